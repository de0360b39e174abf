"""Benchmark of the compressed Coulomb-integral engine on one GB300 (one JSON line).

Workload (the paper's 9171-planewave scale): cutoff |n| <= 13 (Nb = 9171 planewaves),
L = 20 bohr, 64 quadrature nodes (58 kept), Fermi radius 8 (Mocc = 2109).  One step is
one pass of the whole hot path over one batch of synthetic input:
  1. reconstruct 1e8 seeded momentum-conserving quadruples (IJ|KL)  (8 B of uint16 basis
     ids in, 4 B out each; the int32-id and int8x4-vector forms, 16 B each, are timed in
     the breakdown)
  2. all Nb^2 = 8.41e7 exchange-type pair integrals V(k_i - k_j)
  3. exchange sums eps(k) on the (2R+1)^3 grid and E_x by Toeplitz mode products
     (plain FP32 path; mixed bf16x3 path as well when --mixed), FP64 E_x reduction.
metric value = Coulomb evaluations per second = (1e8 + Nb^2 + Nb * Mocc) / step time,
the exchange counted as the Nb * Mocc pair evaluations its sums replace.
Inputs (0.8 GB of uint16-id quadruples) are larger than L2 (129 MB), so no flush is needed.

--impl reference times the FP64 CPU oracle (the slow, plainly correct restatement of the
paper) on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

R, L, S, R_F = 13, 20.0, 64, 8
N_QUADS = 100_000_000
# ncu DRAM bytes (read + written) of a 2e7-quadruple k_col launch of the current kernel, per
# quadruple encoding (only the encoding that was captured; the others report null)
TRAFFIC_2E7 = {"ids16": 201.3e6}
METRIC = "pair-Coulomb evals/s and integrals/s on 1 GB300, mixed vs FP32 at <=1e-4 rel err"
UNIT = "Coulomb evals/s"
WORKLOAD = ("paper scale: |n|<=13 (9171 planewaves), L=20 bohr, 64 nodes, R_F=8 (2109 occ); "
            "1e8 conserving quadruples + all 9171^2 pairs + exchange sums")


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.p = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
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
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _bf16_peak():
    """Dense bf16 tensor peak (TFLOP/s): the measured cuBLAS burst figure, else the
    fallback measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def _sig(x, n=4):
    """x rounded to n significant digits (compact JSON)."""
    if x is None or x == 0 or not np.isfinite(x):
        return x
    return float(f"{x:.{n}g}")


# ------------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import coulomb_inputs as ci
    import paper_1502_08043_gb300 as cc
    from paper_1502_08043_gb300 import replicas

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream(dev)

    t = cc.build_tables("periodic", R=R, L=L, S=S)
    Nb, Mg = t.info["Nb"], t.info["Mg"]
    Mocc = 2109
    n = args.quads
    # every rank owns its own slice of the quadruple stream (weak scaling, no collective)
    qid = torch.empty((n, 4), dtype=torch.int32, device=dev)
    first, _ = replicas.quad_slice(rank, n)
    ci.quads_device(R, first, n, qid)
    # three encodings of the same quadruples: uint16 basis ids (8 B, needs Nb <= 65536),
    # int32 ids (16 B) and the int8x4 vectors (16 B); the step reads --quad-format, the
    # other two are timed in the breakdown
    forms = {"ids": qid,
             "vec": torch.from_numpy(cc.basis(R)).to(dev)[qid.long().view(-1)].view(n, 4, 4)}
    if Nb <= 65536:
        forms["ids16"] = torch.where(qid >= 32768, qid - 65536, qid).to(torch.int16)
    q = forms[args.quad_format]
    qbytes = q.element_size() * q[0].numel()   # bytes per quadruple
    vals = torch.empty(n, dtype=torch.float32, device=dev)
    pairs = torch.empty((Nb, Nb), dtype=torch.float32, device=dev)
    eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
    eps_mx = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
    Ex = torch.empty(2, dtype=torch.float64, device=dev)
    Ex_mx = torch.empty(2, dtype=torch.float64, device=dev)
    lookup = args.lookup
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]

    def step(k=None):
        if k is not None:
            ev[k][0].record(st)
        cc.reconstruct_integrals(t, q, vals, lookup=lookup)
        if k is not None:
            ev[k][1].record(st)
        cc.pair_matrix(t, 0, Nb, pairs, lookup=lookup)
        cc.exchange_sums(t, R_F, eps, Ex, precision="fp32")
        if args.mixed:
            cc.exchange_sums(t, R_F, eps_mx, Ex_mx, precision="bf16x3")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = local
    clocks = Clocks(gpu_id)
    clocks.start()
    # keep the GPU under the same load for a second before the timed steps so that the
    # 200 ms clock sampler sees the loaded state (these steps are not timed)
    tb = time.perf_counter()
    while time.perf_counter() - tb < 1.0:
        step()
        torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(st)
    for k in range(args.steps):
        step(k)
    t1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    k_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ms = replicas.max_over_ranks(ms, dev)

    # per-part timing (outside the timed region; for the breakdown only)
    def time_it(fn, reps=5):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        fn()
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    parts = {
        "reconstruct_ms": k_ms,
        "pairs_ms": time_it(lambda: cc.pair_matrix(t, 0, Nb, pairs, lookup=lookup)),
        "exchange_fp32_ms": time_it(lambda: cc.exchange_sums(t, R_F, eps, Ex, precision="fp32")),
    }
    other = "separable" if lookup == "collapsed" else "collapsed"
    parts[f"reconstruct_{other}_ms"] = time_it(
        lambda: cc.reconstruct_integrals(t, q, vals, lookup=other))
    for fname, qo in forms.items():
        if fname != args.quad_format:
            parts[f"reconstruct_{lookup}_{fname}_ms"] = time_it(
                lambda qo=qo: cc.reconstruct_integrals(t, qo, vals, lookup=lookup))
    if args.mixed:
        parts["exchange_bf16x3_ms"] = time_it(
            lambda: cc.exchange_sums(t, R_F, eps_mx, Ex_mx, precision="bf16x3"))

    evals = n + Nb * Nb + Nb * Mocc
    value = replicas.job_throughput(evals, world, ms)

    # end to end through the public API with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        hq = torch.empty(tuple(q.shape), dtype=q.dtype, pin_memory=True)
        hq.copy_(q.cpu())
        hv = torch.empty(n, dtype=torch.float32, pin_memory=True)
        hp = torch.empty((Nb, Nb), dtype=torch.float32, pin_memory=True)
        he = torch.empty(Mg ** 3, dtype=torch.float32, pin_memory=True)
        hx = torch.empty(2, dtype=torch.float64, pin_memory=True)

        # the step through the public API with host buffers: the pair matrix and the
        # exchange sums (which need no quadruples) are computed first and go down on one
        # copy stream while the quadruples come up in chunks on another; each chunk is
        # reconstructed as soon as it has landed and its values follow the pairs down
        # (H2D, compute and D2H overlap; the link carries both directions at once)
        nchunk = args.e2e_chunks
        bounds = [n * c // nchunk for c in range(nchunk + 1)]
        up = torch.cuda.Stream(dev)
        down = torch.cuda.Stream(dev)
        loaded = [torch.cuda.Event() for _ in range(nchunk)]
        done = [torch.cuda.Event() for _ in range(nchunk)]
        ev_head = torch.cuda.Event()

        def e2e_step():
            up.wait_stream(st)      # the previous step has finished with q
            down.wait_stream(st)    # ... and with the host result buffers
            with torch.cuda.stream(up):
                for c in range(nchunk):
                    a, b = bounds[c], bounds[c + 1]
                    q[a:b].copy_(hq[a:b], non_blocking=True)
                    loaded[c].record(up)
            cc.pair_matrix(t, 0, Nb, pairs, lookup=lookup, stream=st)
            cc.exchange_sums(t, R_F, eps, Ex, precision="fp32", stream=st)
            ev_head.record(st)
            with torch.cuda.stream(down):
                down.wait_event(ev_head)
                hp.copy_(pairs, non_blocking=True)
                he.copy_(eps, non_blocking=True)
                hx.copy_(Ex, non_blocking=True)
            for c in range(nchunk):
                a, b = bounds[c], bounds[c + 1]
                st.wait_event(loaded[c])
                cc.reconstruct_integrals(t, q[a:b], vals[a:b], lookup=lookup, stream=st)
                done[c].record(st)
                with torch.cuda.stream(down):
                    down.wait_event(done[c])
                    hv[a:b].copy_(vals[a:b], non_blocking=True)
            st.wait_stream(down)
            st.wait_stream(up)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        ks = max(2, min(args.steps, 5))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(ks):
            e2e_step()
        b.record(st)
        torch.cuda.synchronize()
        ems = a.elapsed_time(b) / ks
        ems = replicas.max_over_ranks(ems, dev)
        e2e = {"value": replicas.job_throughput(evals, world, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(n * qbytes),
               "d2h_bytes_per_step": int(n * 4 + Nb * Nb * 4 + Mg ** 3 * 4 + 16),
               "ms_per_step": ems}

    peak, peak_kind = _peaks()
    # ncu DRAM bytes (read + written) of one k_col launch for 2e7 quadruples, per quadruple
    # encoding (TRAFFIC_2E7), scaled by the quadruples of this launch
    if args.traffic is None and lookup == "collapsed":
        args.traffic = TRAFFIC_2E7.get(args.quad_format)
        args.traffic = None if args.traffic is None else args.traffic * n / 2e7
    algo_bytes = float(qbytes + 4) * n    # the quadruple in, one FP32 value out
    if lookup == "collapsed":
        achieved = algo_bytes / (k_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": args.traffic,
                    "kernel": f"k_col ({args.quad_format} quadruples)",
                    "algorithmic_bytes_per_launch": algo_bytes, "peak_source": peak_kind,
                    "traffic_source": "ncu dram bytes of a 2e7-quadruple launch, scaled"}
    else:
        achieved = algo_bytes / (k_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": args.traffic, "kernel": "k_sep",
                    "algorithmic_bytes_per_launch": algo_bytes, "peak_source": peak_kind}

    n_launch = 2 + 8 + (args.mixed_launches if args.mixed else 0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded SplitMix64 quadruples; shell-closed Fermi sphere)",
        "config": {"workload": WORKLOAD, "R": R, "L_bohr": L, "S": S,
                   "S_eff": t.info["S_eff"], "R_F": R_F, "Nb": Nb, "Mocc": Mocc,
                   "quadruples": n, "quad_format": args.quad_format, "pairs": Nb * Nb,
                   "lookup": lookup,
                   "evals_per_step": evals, "l2_policy": f"inputs larger than L2 ({n * qbytes / 1e9:.1f} GB of quadruples)",
                   "parallelism": f"replicas x{world} (independent quadruple slices)"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": n_launch * args.steps,
        "clocks": clk, "breakdown": parts,
        "rates": {"integrals_per_s": n / (k_ms * 1e-3),
                  "pairs_per_s": Nb * Nb / (parts["pairs_ms"] * 1e-3)},
    }
    if rank == 0 and world == 1 and args.mode_products:
        line["mode_products"] = {n: mode_products(n, with_fp16=True)
                                 for n in args.mode_products.split(",")}
    if rank == 0 and world == 1 and not args.no_extras:
        line["batched"] = batched()
        line["large_lookups"] = large_lookups()
        line["general_lookups"] = general_lookups()
        line["paper_replay"] = paper_replay()
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    if rank == 0 and world == 1:
        # last on the line: the metric's mixed-vs-FP32 comparison in compact form
        try:
            line["mixed_vs_fp32"] = mixed_vs_fp32(line.get("mode_products"),
                                                  line.get("large_lookups"),
                                                  line.get("batched"),
                                                  line.get("general_lookups"))
        except (KeyError, TypeError, ValueError) as e:   # never lose the line to a summary
            line["mixed_vs_fp32"] = {"error": f"summary not formed: {e!r}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    t.free()
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- mode products: FP32 vs mixed
MP_CONFIGS = {"precision": (31, 40.0, 96, 20), "large": (63, 60.0, 128, 40)}


def tc_slab_executed_flop(R, R_F, Mg, S_eff, periodic=True):
    """Flop the tensor-core exchange issues for one call.  Grid sides up to 64 (the small-grid
    kernel, two slabs per 128-row MMA): per (slab pair, node) unit, MMA1 and MMA2 of
    3 x 2 x 128 x N2 x 16 per K step over the band, plus the A term 2 x 2 x 128 x N2 x 16 per
    h step (periodic).  Larger grids (the 128-row slab kernel): per unit and slab, MMA1
    (3 x 128 x B x B), MMA2 (3 x 128 x B x N2) and, when the A term runs on the tensor cores
    (periodic, band B <= 96), 2 x 128 x B x 16 nh.  B = the band rounded out to 16-column
    pieces, N2 = the grid side rounded up to 16, nh = ceil((R_F + 1) / 16)."""
    N2 = (Mg + 15) & ~15
    nh = (R_F + 16) >> 4
    if Mg <= 64:
        steps = (min(64, (R + R_F + 16) & ~15) - ((R - R_F) & ~15)) // 16
        per_unit = 2 * 128 * N2 * 16 * (6 * steps + (2 * nh if periodic else 0))
        return per_unit * ((Mg + 1) // 2) * S_eff
    B = ((R + R_F + 16) & ~15) - ((R - R_F) & ~15)
    per_slab = 2 * 128 * (3 * B * B + 3 * B * N2 + (2 * B * 16 * nh if periodic and B <= 96 else 0))
    return per_slab * 2 * ((Mg + 1) // 2) * S_eff


def simt_slab_flop(R_F, Mg, S_eff):
    """Flop of the SIMT slab algorithm: per (slab, node), U = T[:, band] R' (Mg x nb x nb)
    and E += U T[band, :] (Mg x nb x Mg), nb = 2 R_F + 1."""
    nb = 2 * R_F + 1
    return 2.0 * Mg * nb * (nb + Mg) * Mg * S_eff


def mode_products(name, reps=10, oracle_sample=200, with_fp16=True):
    """Exchange sums of one single-box workload by the plain FP32 SIMT path (the slab
    algorithm, and the dense GEMM chain over the full grid), and by the bf16x3 and fp16x3
    tensor-core slab kernel: device time per call (CUDA events, inputs resident), useful
    flop rate 6 Mg^4 S_eff, executed tensor flop rate, and the accuracy of each against the
    FP64 oracle on a seeded sample of basis functions."""
    import torch

    import paper_1502_08043_gb300 as cc
    R, L, S, R_F = MP_CONFIGS[name]
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev)
    t = cc.build_tables("periodic", R=R, L=L, S=S)
    Mg, S_eff = t.info["Mg"], t.info["S_eff"]
    out = {"R": R, "L_bohr": L, "S": S, "S_eff": S_eff, "R_F": R_F, "Mg": Mg}
    peak, peak_kind = _bf16_peak()
    res = {}
    precs = ["fp32", "fp32_dense", "bf16x3"] + (["fp16x3"] if with_fp16 else [])
    for prec in precs:
        eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
        Ex = torch.empty(2, dtype=torch.float64, device=dev)
        p = "fp32" if prec == "fp32_dense" else prec
        cc.lib().cc_set_simt_variant(1 if prec == "fp32_dense" else 0)
        if prec == "fp32_dense":   # the chain at its autotuned tiles
            out["fp32_dense_tiles"] = cc.autotune_gemm(t, R_F, precision="fp32", reps=2)
        try:
            n = max(2, reps // 4) if prec == "fp32_dense" else reps
            for _ in range(2):
                cc.exchange_sums(t, R_F, eps, Ex, precision=p)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            for _ in range(n):
                cc.exchange_sums(t, R_F, eps, Ex, precision=p)
            b.record(st)
            torch.cuda.synchronize()
        finally:
            cc.lib().cc_set_simt_variant(0)
        ms = a.elapsed_time(b) / n
        res[prec] = (ms, eps.cpu().numpy().astype(np.float64), float(Ex[0].item()))
        out[prec + "_ms"] = ms
        out[prec + "_useful_tflops"] = 6.0 * Mg ** 4 * S_eff / (ms * 1e-3) / 1e12
    # the same tensor-core product without the lo-plane correction (hi * hi only)
    cc.lib().cc_set_mixed_terms(1)
    try:
        eps = torch.empty(Mg ** 3, dtype=torch.float32, device=dev)
        Ex = torch.empty(2, dtype=torch.float64, device=dev)
        for _ in range(2):
            cc.exchange_sums(t, R_F, eps, Ex, precision="bf16x3")
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            cc.exchange_sums(t, R_F, eps, Ex, precision="bf16x3")
        b.record(st)
        torch.cuda.synchronize()
        res["bf16x1"] = (a.elapsed_time(b) / reps, eps.cpu().numpy().astype(np.float64),
                         float(Ex[0].item()))
        out["bf16x1_ms"] = res["bf16x1"][0]
        out["bf16x1_note"] = "bf16 hi * hi products only (no lo-plane correction)"
    finally:
        cc.lib().cc_set_mixed_terms(3)
    out["fp32_executed_tflops"] = simt_slab_flop(R_F, Mg, S_eff) / (res["fp32"][0] * 1e-3) / 1e12
    ex = tc_slab_executed_flop(R, R_F, Mg, S_eff)
    for prec in ("bf16x3", "fp16x3") if with_fp16 else ("bf16x3",):
        out[prec + "_executed_tflops"] = ex / (res[prec][0] * 1e-3) / 1e12
        out[prec + "_useful_frac_of_peak"] = out[prec + "_useful_tflops"] / peak
        out[prec + "_executed_frac_of_peak"] = out[prec + "_executed_tflops"] / peak
    out["bf16_peak_tflops"] = peak
    out["peak_source"] = peak_kind + " bf16 burst (MEASURED_PEAKS.json)"
    out["speedup_bf16x3_vs_fp32"] = res["fp32"][0] / res["bf16x3"][0]
    out["speedup_bf16x3_vs_fp32_dense"] = res["fp32_dense"][0] / res["bf16x3"][0]
    out["speedup_fp32_vs_fp32_dense"] = res["fp32_dense"][0] / res["fp32"][0]
    if with_fp16:
        out["speedup_fp16x3_vs_fp32"] = res["fp32"][0] / res["fp16x3"][0]
    if oracle_sample:
        from oracle import basis as ob
        from oracle import exchange as ox
        from oracle import quadrature as oq
        n_sub, q_tail = oq.default_periodic_mesh(S, R)
        aa, ww, _ = oq.laplace_mesh(S, n_sub, q_tail)
        keep = oq.prune_periodic(aa, ww, R, 1e-9)
        Nb = ob.count(R)
        idx = np.unique(np.random.default_rng(7).integers(0, Nb, oracle_sample))
        ref = ox.eps_separable(R, R_F, L, aa[keep], ww[keep], k_idx=idx)
        k = ob.basis(R)[idx] + R
        flat = (k[:, 0] * Mg + k[:, 1]) * Mg + k[:, 2]
        for prec in precs + ["bf16x1"]:
            got = res[prec][1][flat]
            out[prec + "_max_rel_err_vs_oracle"] = float(np.max(np.abs(got - ref) / np.abs(ref)))
        out["oracle_sample"] = f"{len(idx)} seeded basis functions of {Nb}"
    t.free()
    return out


def mixed_vs_fp32(mp, large, batched_sec, general):
    """The metric's mixed-vs-FP32 comparison in a compact form (the end of the JSON line):
    per single-box workload the FP32 times (slab algorithm and dense chain), the bf16x3 and
    fp16x3 times, tensor fractions of the measured bf16 peak (useful 6 Mg^4 S flop and
    executed flop), errors against the FP64 oracle, speedups at equal stated accuracy."""
    out = {}
    for name, tag in (("precision", "cfg3_grid63"), ("large", "cfg5_grid127")):
        m = mp.get(name) if mp else None
        if not m:
            continue
        out[tag] = {
            "ms": {k: _sig(m.get(k + "_ms")) for k in ("fp32", "fp32_dense", "bf16x3", "fp16x3")},
            "bf16x3_frac_useful": _sig(m.get("bf16x3_useful_frac_of_peak"), 3),
            "bf16x3_frac_exec": _sig(m.get("bf16x3_executed_frac_of_peak"), 3),
            "fp32_exec_tflops": _sig(m.get("fp32_executed_tflops"), 3),
            "err": {k: _sig(m.get(k + "_max_rel_err_vs_oracle"), 2)
                    for k in ("fp32", "bf16x3", "fp16x3", "bf16x1")},
            "x_bf16x3_vs_fp32": _sig(m.get("speedup_bf16x3_vs_fp32"), 3),
            "x_bf16x3_vs_fp32_dense": _sig(m.get("speedup_bf16x3_vs_fp32_dense"), 3),
        }
    if batched_sec:
        out["batch256_ms"] = {k: _sig(batched_sec[k]["ms_per_batch"]) for k in ("fp32", "bf16x3", "fp64")
                              if k in batched_sec}
        out["batch256_bf16x3_frac_exec"] = _sig(batched_sec["bf16x3"].get("executed_frac_of_peak"), 3)
    if large:
        out["cfg5_1e9_lookups"] = {k: {"ms": _sig(v.get("ms")), "hbm_frac": _sig(v.get("hbm_frac"), 3)}
                                   for k, v in large.items() if isinstance(v, dict) and "hbm_frac" in v}
        tuned = large.get("vec_separable_mesh_for_1e-8")
        if tuned:
            out["cfg5_separable_mesh_for_1e-8"] = {
                "ms": _sig(tuned["ms"]), "S_eff": tuned["S_eff"],
                "x_vs_128_node_mesh": _sig(tuned["speedup_vs_128_node_mesh"], 3)}
    if general:
        out["general_box_lookups"] = {"integrals_per_s": _sig(general["fp32"]["integrals_per_s"]),
                                      "fp64_integrals_per_s": _sig(general["fp64"]["integrals_per_s"])}
    return out


# ---------------------------------------------------------------- batched boxes, large lookups
def batched(reps=10):
    """256 boxes (|n| in 4..24, L in 8..30 bohr, R_F 0.4-0.8 of the cutoff, 16..96 nodes) in
    one persistent graph-captured launch: autotuned launch shape, device time per batch."""
    import torch

    import coulomb_inputs as ci
    import paper_1502_08043_gb300 as cc
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev)
    boxes = ci.box_params(256)
    B = cc.Batch(boxes)
    out = {"boxes": len(boxes), "grid_points": int(B.offsets[-1])}
    pairs = sum(b_pair(b) for b in boxes)
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64), ("bf16x3", torch.float32)):
        eps = torch.empty(int(B.offsets[-1]), dtype=dt, device=dev)
        Ex = torch.empty((B.nbox, 2), dtype=torch.float64, device=dev)
        choice = B.tune(eps, Ex, reps=3, precision=prec)
        B.exchange(eps, Ex, precision=prec)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            B.exchange(eps, Ex, precision=prec)
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out[prec] = {"ms_per_batch": ms, "boxes_per_s": len(boxes) / (ms * 1e-3),
                     "pair_evals_per_s": pairs / (ms * 1e-3), "tuned": choice,
                     "work_items": B.n_items}
    out["pair_evals_per_batch"] = pairs
    peak, peak_kind = _bf16_peak()
    infos = [cc.build_tables("periodic", R=b["R"], L=b["L"], S=b["S"]) for b in boxes]
    ex = sum(tc_slab_executed_flop(b["R"], b["R_F"], 2 * b["R"] + 1, t.info["S_eff"])
             for b, t in zip(boxes, infos))
    useful = sum(6.0 * (2 * b["R"] + 1) ** 4 * t.info["S_eff"] for b, t in zip(boxes, infos))
    for t in infos:
        t.free()
    ms = out["bf16x3"]["ms_per_batch"]
    out["bf16x3"]["executed_tflops"] = ex / (ms * 1e-3) / 1e12
    out["bf16x3"]["useful_tflops"] = useful / (ms * 1e-3) / 1e12
    out["bf16x3"]["executed_frac_of_peak"] = out["bf16x3"]["executed_tflops"] / peak
    out["bf16x3"]["useful_frac_of_peak"] = out["bf16x3"]["useful_tflops"] / peak
    out["bf16x3"]["kernel"] = "small-grid tensor-core kernel, every box in one launch"
    B.free()
    return out


# ---------------------------------------------------------------- paper replay: Table I, Fig. 1
def _e_ks(M, L):
    """Kohn-Sham exchange of M electrons per spin in a cube of side L, -(3/4)(6/pi)^(1/3)
    M^(4/3) / L (Sec. III)."""
    return -0.75 * (6.0 / np.pi) ** (1.0 / 3.0) * M ** (4.0 / 3.0) / L


def _n_occupied(R_F):
    """Integer vectors with |n|^2 <= R_F^2 (the occupied states of one spin)."""
    r = np.arange(-R_F, R_F + 1)
    return int(((r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2)
                <= R_F * R_F).sum())


def _exchange_timed(t, R_F, prec, reps):
    import torch
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev)
    Mg = t.info["Mg"]
    eps = torch.empty(Mg ** 3, dtype=torch.float64 if prec == "fp64" else torch.float32,
                      device=dev)
    Ex = torch.empty(2, dtype=torch.float64, device=dev)
    import paper_1502_08043_gb300 as cc
    cc.exchange_sums(t, R_F, eps, Ex, precision=prec)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(reps):
        cc.exchange_sums(t, R_F, eps, Ex, precision=prec)
    b.record(st)
    torch.cuda.synchronize()
    return float(Ex[0].item()), a.elapsed_time(b) / reps


def paper_replay(reps=5):
    """Table I (M = 9171 parallel-spin electrons, L = 2 bohr, finite-box kernel, both meshes
    of the paper) through the GPU box-kernel mode products in FP64, FP32 and bf16x3, each
    ratio E_x / E_KS against the printed total; and Fig. 1 (E_x / E_KS against M^(-1/3) for
    R_F = 1 .. 13, periodic kernel, |n| <= 13, L = 10, 64-node default mesh) with its
    extrapolation to M -> infinity, which the paper puts at 1."""
    import paper_1502_08043_gb300 as cc
    rows = []
    here = os.path.dirname(os.path.abspath(__file__))
    for line in open(os.path.join(here, "tests", "golden", "table1.txt")):
        if line.strip() and not line.startswith("#"):
            mesh, par, _, total = line.split()
            rows.append((mesh, int(par), float(total)))
    ks = _e_ks(9171, 2.0)
    table = []
    for mesh, par, total in rows:
        if mesh == "mesh1":
            t = cc.build_tables("box", R=13, L=2.0, S=2 * par, n_sub=0, q_tail=par)
        else:
            t = cc.build_tables("box", R=13, L=2.0, S=8 * par + 90, n_sub=7, q_tail=90)
        row = {"mesh": mesh, "param": par, "S": t.info["S_eff"], "paper_total": total}
        for prec in ("fp64", "fp32", "bf16x3"):
            ex, ms = _exchange_timed(t, 13, prec, reps)
            row[prec] = ex / ks
            row[prec + "_dev"] = ex / ks - total
            row[prec + "_ms"] = ms
        table.append(row)
        t.free()
    t = cc.build_tables("periodic", R=13, L=10.0, S=64)
    fig = {"R_F": [], "M": [], "ratio_fp64": [], "ms_fp64": []}
    for R_F in range(1, 14):
        ex, ms = _exchange_timed(t, R_F, "fp64", reps)
        M = _n_occupied(R_F)
        fig["R_F"].append(R_F)
        fig["M"].append(M)
        fig["ratio_fp64"].append(ex / _e_ks(M, 10.0))
        fig["ms_fp64"].append(ms)
    t.free()
    x = np.array(fig["M"], dtype=float) ** (-1.0 / 3.0)
    y = np.array(fig["ratio_fp64"])
    slope = (y[-1] - y[-2]) / (x[-1] - x[-2])
    fig["extrapolated_M_inf"] = float(y[-1] - slope * x[-1])
    fig["note"] = ("two-point linear extrapolation in M^(-1/3) from R_F = 12, 13; "
                   "the paper's Fig. 1 data are not printed, only the trend and limit 1")
    return {"table1": table,
            "table1_max_abs_dev": {p: max(abs(r[p + "_dev"]) for r in table)
                                   for p in ("fp64", "fp32", "bf16x3")},
            "fig1": fig}


def b_pair(b):
    """Pair evaluations an exchange sum of a box replaces: basis size x occupied count."""
    from coulomb_inputs import sphere_vectors
    return len(sphere_vectors(b["R"])) * len(sphere_vectors(b["R_F"]))


def large_lookups(n=1_000_000_000, reps=3):
    """1e9 seeded conserving quadruples at |n| <= 63 (1,047,331 planewaves), FP32 tables in
    shared memory: device time per pass for both table forms."""
    import torch

    import coulomb_inputs as ci
    import paper_1502_08043_gb300 as cc
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev)
    t = cc.build_tables("periodic", R=63, L=60.0, S=128)
    q = torch.empty((n, 4), dtype=torch.int32, device=dev)
    ci.quads_device(63, 0, n, q)
    vals = torch.empty(n, dtype=torch.float32, device=dev)
    out = {"quadruples": n, "S_eff": t.info["S_eff"],
           "note": "ids: the four ids decoded on chip from 128 KB of line hints in shared "
                   "memory; ids_l2gather: 4 basis vectors gathered from the 4.2 MB basis "
                   "table (L2); vec: the quadruple carries its four int8x4 vectors"}
    peak, _ = _peaks()
    # the same quadruples in vector form (16 B each as well)
    vecs = torch.from_numpy(cc.basis(63)).to(dev)[q.long().view(-1)].view(n, 4, 4)
    for fmt, qq, lookups in (("ids", q, ("collapsed", "separable")),
                             ("ids_l2gather", q, ("collapsed",)),
                             ("vec", vecs, ("collapsed", "separable"))):
        cc.lib().cc_set_id_decode(0 if fmt == "ids_l2gather" else 1)
        for lookup in lookups:
            cc.reconstruct_integrals(t, qq, vals, lookup=lookup)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            for _ in range(reps):
                cc.reconstruct_integrals(t, qq, vals, lookup=lookup)
            b.record(st)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            gbs = 20.0 * n / (ms * 1e-3) / 1e9
            out[f"{fmt}_{lookup}"] = {"ms": ms, "integrals_per_s": n / (ms * 1e-3),
                                      "hbm_GBps": gbs, "hbm_frac": gbs / peak}
    cc.lib().cc_set_id_decode(1)
    # the separable lookup on tables built for a stated method error (1e-8): the tuned mesh
    # with the fewest nodes instead of the 128-node workload mesh
    tt = cc.build_tables_for_error("periodic", R=63, L=60.0, target=1e-8)
    cc.reconstruct_integrals(tt, vecs, vals, lookup="separable")
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(reps):
        cc.reconstruct_integrals(tt, vecs, vals, lookup="separable")
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    out["vec_separable_mesh_for_1e-8"] = {
        "ms": ms, "integrals_per_s": n / (ms * 1e-3), "S": tt.info["S"],
        "S_eff": tt.info["S_eff"], "alpha_c": tt.info["alpha_c"], "ratio": tt.info["ratio"],
        "speedup_vs_128_node_mesh": out["vec_separable"]["ms"] / ms}
    tt.free()
    del q, vals, vecs
    t.free()
    torch.cuda.empty_cache()
    return out


def general_lookups(n=20_000_000, reps=5):
    """General (not necessarily momentum-conserving) box-kernel integrals at the paper's
    stored-table case: 9171 planewaves (|n| <= 13), box side 2 bohr, Mesh 1 with Q = 90
    (180 nodes; Sec. III quotes < 2.4 MB of tables for it).  n quadruples of four independent
    uniform ids (almost all non-conserving), generated on the device, uint16 ids.  The
    two-index tables (one row of S_pad node values per canonical (D1, D2) code) exceed
    shared memory, so every integral reads 3 rows through L1: the kernel is bound by L1
    bandwidth (152 SMs x 128 B/clk), not by HBM."""
    import torch

    import coulomb_inputs as ci
    import paper_1502_08043_gb300 as cc
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev)
    t = cc.build_tables("box", R=13, L=2.0, S=180, n_sub=0, q_tail=90)
    info = t.info
    q = torch.empty((n, 4), dtype=torch.int32, device=dev)
    ci.quads_device(13, 0, n, q, stream=ci.STREAM_UNIFORM)
    q16 = torch.where(q >= 32768, q - 65536, q).to(torch.int16)
    del q
    S_pad = 32 * ((info["S_eff"] + 31) // 32)
    nb = 9171
    out = {"quadruples": n, "R": 13, "L_bohr": 2.0, "S_eff": info["S_eff"],
           "codes_per_node": info["general_codes"],
           "paper_entries_per_node_4N23": 4.0 * nb ** (2.0 / 3.0),
           "table_fp64_bytes": 8 * info["general_codes"] * info["S_eff"],
           "table_fp32_lookup_bytes": info["general_table_bytes"],
           "paper_table_bytes_claim": "< 2.4 MB (Sec. III, 9171 planewaves)"}
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = 2.07e9
    for prec, dt, eb in (("fp32", torch.float32, 4), ("fp64", torch.float64, 8)):
        vals = torch.empty(n, dtype=dt, device=dev)
        cc.reconstruct_integrals(t, q16, vals, lookup="general")
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            cc.reconstruct_integrals(t, q16, vals, lookup="general")
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        l1 = 3.0 * S_pad * eb * n / (ms * 1e-3)
        out[prec] = {"ms": ms, "integrals_per_s": n / (ms * 1e-3),
                     "hbm_GBps": (8 + eb) * n / (ms * 1e-3) / 1e9,
                     "l1_table_GBps": l1 / 1e9,
                     "l1_frac": l1 / (sm * 128 * clk)}
        del vals
    out["l1_peak_note"] = f"{sm} SMs x 128 B/clk x 2.07 GHz"
    t.free()
    del q16
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------------------- oracle
def oracle_sample(budget_s: float, part: int = 0):
    """Run the FP64 oracle on a bounded sample of the workload; returns (evals, seconds,
    description).  `part` selects a disjoint slice of the quadruple stream, pair rows and k
    points (one per worker of the all-core baseline)."""
    import coulomb_inputs as ci
    from oracle import exchange as ox
    from oracle import quadrature as oq
    from oracle import reconstruct as orc
    n_sub, q_tail = oq.default_periodic_mesh(S, R)
    a, w, _ = oq.laplace_mesh(S, n_sub, q_tail)
    keep = oq.prune_periodic(a, w, R, 1e-9)
    a, w = a[keep], w[keep]
    Nb, Mocc = 9171, 2109
    chunk_q, chunk_r, chunk_k = 200_000, 20, 64
    q0, r0, k0 = part * 50_000_000, part * 577, part * 4099
    nq, rows, nk = 0, 0, 0
    t0 = time.perf_counter()
    # the same mix as a GPU step: quadruples : pairs : exchange = 1e8 : Nb^2 : Nb Mocc
    while time.perf_counter() - t0 < budget_s:
        q = ci.quads(R, q0 + nq, chunk_q)
        orc.reconstruct(q, R, L, "separable", a=a, w=w)
        nq += chunk_q
        orc.pair_matrix(R, L, rows=np.arange(r0 + rows, r0 + rows + chunk_r) % Nb,
                        value="separable", a=a, w=w)
        rows += chunk_r
        ox.eps_separable(R, R_F, L, a, w, k_idx=np.arange(k0 + nk, k0 + nk + chunk_k) % Nb)
        nk += chunk_k
    dt = time.perf_counter() - t0
    evals = nq + rows * Nb + nk * Mocc
    desc = (f"{nq} quadruples + {rows} pair rows x {Nb} + eps at {nk} k x {Mocc} occupied, "
            f"FP64 numpy node sums (oracle as it stands)")
    return evals, dt, desc


def _oracle_worker(job):
    budget, part = job
    return oracle_sample(budget, part)


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_all_cores(seconds: float):
    """The oracle on every host core at once: one single-threaded worker process per core
    (spawned, numpy pinned to one thread), each on its own slice of the workload for
    `seconds`; value = all evaluations / the slowest worker's time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                           "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(seconds, k) for k in range(cores)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    evals = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    desc = (f"{cores} workers x ({res[0][2]}), each {seconds:.0f} s on its own slice; "
            f"{evals} evaluations in total")
    return evals, dt, desc, cores


def cpu_baseline(seconds=12.0):
    evals, dt, desc, cores = oracle_all_cores(seconds)
    return {"value": evals / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
            "seconds": dt, "cpu_model": _cpu_model(), "nproc": os.cpu_count()}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(0.2)
    tot_e, tot_t, desc, cores = 0, 0.0, "", 1
    for _ in range(args.steps):
        e, dt, desc, cores = oracle_all_cores(args.ref_seconds)
        tot_e += e
        tot_t += dt
    v = tot_e / tot_t
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 quadruples; shell-closed Fermi sphere)",
            "config": {"workload": WORKLOAD, "R": R, "L_bohr": L, "S": S, "R_F": R_F,
                       "lookup": "separable", "parallelism": f"oracle, rank 0 only, {cores} host cores"},
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": desc, "value": v,
                             "unit": UNIT, "cpu_model": _cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PROFILE_CASES = {
    "exchange_grid63": "bf16x3 exchange sums, |n| <= 31, R_F = 20, 96 nodes (3 calls)",
    "exchange_grid127": "bf16x3 then FP32 exchange sums, |n| <= 63, R_F = 40, 128 nodes "
                        "(2 calls each)",
    "batch48": "bf16x3 exchange sums of the first 48 boxes of the batched workload (2 calls)",
    "general2e6": "general box-kernel lookups, 9171 planewaves, 180 nodes, 2e6 uniform-id "
                  "quadruples (3 calls)",
    "col_ids16_2e7": "collapsed lookups of 2e7 uint16-id quadruples, |n| <= 13 (3 calls)",
    "col_ids_1e8": "collapsed lookups of 1e8 int32-id quadruples, |n| <= 63, ids decoded on "
                   "chip (3 calls)",
}


def profile_case(name):
    """One small, fixed invocation of a hot-path kernel for an ncu capture (a few launches,
    a few GB on the device at most); prints what ran.  No timing."""
    import torch

    import coulomb_inputs as ci
    import paper_1502_08043_gb300 as cc
    dev = torch.device("cuda:0")
    if name == "exchange_grid63":
        t = cc.build_tables("periodic", R=31, L=40.0, S=96)
        eps = torch.empty(63 ** 3, dtype=torch.float32, device=dev)
        Ex = torch.empty(2, dtype=torch.float64, device=dev)
        for _ in range(3):
            cc.exchange_sums(t, 20, eps, Ex, precision="bf16x3")
    elif name == "exchange_grid127":
        t = cc.build_tables("periodic", R=63, L=60.0, S=128)
        eps = torch.empty(127 ** 3, dtype=torch.float32, device=dev)
        Ex = torch.empty(2, dtype=torch.float64, device=dev)
        for prec in ("bf16x3", "fp32"):
            for _ in range(2):
                cc.exchange_sums(t, 40, eps, Ex, precision=prec)
    elif name == "batch48":
        B = cc.Batch(ci.box_params(48))
        eps = torch.empty(int(B.offsets[-1]), dtype=torch.float32, device=dev)
        Ex = torch.empty((B.nbox, 2), dtype=torch.float64, device=dev)
        for _ in range(2):
            B.exchange(eps, Ex, precision="bf16x3")
    elif name == "general2e6":
        t = cc.build_tables("box", R=13, L=2.0, S=180, n_sub=0, q_tail=90)
        n = 2_000_000
        q = torch.empty((n, 4), dtype=torch.int32, device=dev)
        ci.quads_device(13, 0, n, q, stream=ci.STREAM_UNIFORM)
        q16 = torch.where(q >= 32768, q - 65536, q).to(torch.int16)
        out = torch.empty(n, dtype=torch.float32, device=dev)
        for _ in range(3):
            cc.reconstruct_integrals(t, q16, out, lookup="general")
    elif name in ("col_ids16_2e7", "col_ids_1e8"):
        R, n = (13, 20_000_000) if name == "col_ids16_2e7" else (63, 100_000_000)
        t = cc.build_tables("periodic", R=R, L=20.0 if R == 13 else 60.0,
                            S=64 if R == 13 else 128)
        q = torch.empty((n, 4), dtype=torch.int32, device=dev)
        ci.quads_device(R, 0, n, q)
        if R == 13:
            q = torch.where(q >= 32768, q - 65536, q).to(torch.int16)
        out = torch.empty(n, dtype=torch.float32, device=dev)
        for _ in range(3):
            cc.reconstruct_integrals(t, q, out, lookup="collapsed")
    else:
        raise SystemExit(f"unknown profile case {name!r}: one of {sorted(PROFILE_CASES)}")
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "what": PROFILE_CASES[name]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--lookup", default="collapsed", choices=["collapsed", "separable"])
    ap.add_argument("--quads", type=int, default=N_QUADS)
    ap.add_argument("--quad-format", default="ids16", choices=["ids16", "vec", "ids"])
    ap.add_argument("--mixed", action="store_true")
    ap.add_argument("--mixed-launches", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="quadruple chunks the end-to-end step pipelines its copies over")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=2.0)
    ap.add_argument("--mode-products", default="precision,large",
                    help="also time FP32 vs bf16x3 exchange mode products at these single-box "
                         "workloads (precision: |n|<=31, large: |n|<=63); '' to skip")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-boxes and 1e9-lookup sections of the JSON line")
    ap.add_argument("--mp-only", default=None,
                    help="only run the mode-product comparison of this workload, print it")
    ap.add_argument("--batched-only", action="store_true",
                    help="only run the 256-box batched section, print it")
    ap.add_argument("--general-only", action="store_true",
                    help="only run the general box-integral lookup section, print it")
    ap.add_argument("--replay-only", action="store_true",
                    help="only run the Table I / Fig. 1 replay through the GPU path, print it")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one small fixed invocation of a hot-path kernel (for ncu), "
                         "print what ran")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_case:
        profile_case(args.profile_case)
    elif args.mp_only:
        print(json.dumps({"mode_products": mode_products(args.mp_only, oracle_sample=0)}))
    elif args.replay_only:
        print(json.dumps({"paper_replay": paper_replay()}))
    elif args.batched_only:
        print(json.dumps({"batched": batched()}))
    elif args.general_only:
        print(json.dumps({"general_lookups": general_lookups()}))
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
