"""Benchmark: encrypted ensemble Argmax at N = 2^16 on one GB300 (or N ranks,
one per GPU, each with its own independent query mix: weak scaling, no
collective on the data path).

One step = aggregation + encrypted Argmax (SecPE Sec. 3.1 step 3, Alg. 1)
of every query of the mix, batched (secpe_argmax_batch): every homomorphic
operation (NTT, key switching, rescale, rotation, Sign, Max, refresh) runs in
the library's CUDA kernels.  Inputs are encrypted logit ciphertexts resident
in HBM before the timed region (57 GB at 256 queries: larger than L2).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (a bounded sample per step) and prints the same line with
"impl": "reference".
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted ensemble-Argmax/s at N=2^16, batched vs plain; keyswitch GB/s; p99"
# DRAM bytes per algorithmic byte of the N = 2^16 transform-pass family
# (plain NTT/INTT passes, base-conversion pass A, inner-product and
# epilogue passes B), measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) over every family launch of one HMult + relinearise
# + rescale of 8 ciphertexts at level 23 (q0 + 23 x 50-bit, 8 special primes,
# dnum = 3): 2.818 GB of DRAM traffic against 3.045 GB algorithmic.  The
# step's family launches are the same kernels on more items, so their
# traffic is taken in the same proportion to their algorithmic bytes.
NTT16_DRAM_PER_ALG_BYTE = 2.818 / 3.045
ROT_STEPS = [-2, -4, -8, -16, -64, 1, 2, 4, 8, 16, 32]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--queries", type=int, default=256)
    ap.add_argument("--classes", default="2,3,4,6,14,64",
                    help="class counts C drawn uniformly per query (the default is the mix)")
    ap.add_argument("--plain-queries", type=int, default=16,
                    help="queries timed on the one-query-per-launch path")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--kprof", default="ntt16",
                    help="kernel class timed live for the roofline")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the direct secpe_argmax_batch call instead of the captured graph")
    ap.add_argument("--breakdown", action="store_true",
                    help="after the timed steps, one more step with every launch timed by kernel name")
    ap.add_argument("--micro", action="store_true",
                    help="primitive micro-benchmark (N=2^16, 24+4 primes, dnum=3) instead of the Argmax step")
    ap.add_argument("--micro-ops", default="ntt,keyswitch,hmult,rescale,rotate")
    ap.add_argument("--micro-batch", default="1,8,64")
    ap.add_argument("--micro-probe", default="", choices=["", "hmult", "keyswitch", "ntt"],
                    help="after timing, one more call of this op inside the NVTX range 'micro_probe' with the "
                         "--kprof class profiled (its algorithmic bytes, for DRAM-traffic captures)")
    ap.add_argument("--tc-identity-count", type=int, default=10000,
                    help="seeded random ciphertexts of the precision variant's bit-identity checks")
    ap.add_argument("--serve", action="store_true",
                    help="serving loop: Poisson arrivals, continuous batching, p50/p99 latency")
    ap.add_argument("--rates", default="50,200,500,1000,2000")
    ap.add_argument("--serve-queries", type=int, default=384, help="queries submitted per arrival rate")
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--tenants", type=int, default=1,
                    help="serving: tenants with their own resident key sets (queries batch within a tenant)")
    ap.add_argument("--params", default="argmax8", choices=["argmax", "argmax8"],
                    help="Argmax parameter set: argmax8 (8 special 60-bit primes, dnum=3; the default) or "
                         "argmax (4 special, dnum=6)")
    ap.add_argument("--micro-params", default="micro", choices=["micro", "argmax", "argmax8"],
                    help="micro: 24+4 primes, dnum=3 (primitive config); argmax: the Argmax set (dnum=6)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif args.impl == "ours":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x, device="cuda"):
    """Max of a per-rank scalar (timing): the only collective, off the data path."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_queries(n_queries, rank, c_choices=(2, 3, 4, 6, 14, 64)):
    """Each rank serves its own independent query mix (weak scaling: the work
    per GPU is fixed as ranks are added; no data crosses ranks)."""
    from paper_2502_00847_gb300 import workloads
    return workloads.argmax_queries(n_queries, seed=4 + 1000 * rank, C_choices=tuple(c_choices))


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle
def _oracle_copy(job):
    """One copy of the oracle sample: full-size HMult+relin+rescale at levels
    23/15/7 and one rotation at level 12 (single thread)."""
    params_name, seed, seconds_budget = job
    import numpy as np
    from oracle import PRESETS, Oracle
    o = Oracle(PRESETS[params_name])
    t0 = time.perf_counter()
    o.keygen(11 + seed, rot_steps=[1])
    rng = np.random.default_rng(seed)
    a = o.encrypt(rng.uniform(-1, 1, 8), seed=1 + seed)
    samples = []
    for lv in (23, 15, 7):
        x = o.drop(a, lv)
        t = time.perf_counter()
        o.mul(x, x)
        samples.append(time.perf_counter() - t)
        if time.perf_counter() - t0 > seconds_budget:
            break
    t = time.perf_counter()
    o.rotate(o.drop(a, 12), 1)
    t_rot = time.perf_counter() - t
    return sum(samples) / len(samples), t_rot


def oracle_sample(params_name, seconds_budget=20.0, workers=None):
    """Times the CPU oracle on full-size primitives of the workload: one copy
    per host core (at most 16) runs concurrently in a process pool started
    with spawn, so the per-copy times include the contention of a fully
    loaded host.  Returns (HMult seconds, rotation seconds, wall seconds,
    cores used)."""
    import multiprocessing
    n = workers or max(1, min(16, os.cpu_count() or 1))
    t0 = time.perf_counter()
    jobs = [(params_name, i, seconds_budget) for i in range(n)]
    if n == 1:
        res = [_oracle_copy(jobs[0])]
    else:
        with multiprocessing.get_context("spawn").Pool(n) as pool:
            res = pool.map(_oracle_copy, jobs)
    t_mul = sum(r[0] for r in res) / n
    t_rot = sum(r[1] for r in res) / n
    return t_mul, t_rot, time.perf_counter() - t0, n


def op_mix_per_query(queries, reserve_params=None):
    """Keyswitch-equivalent op counts of the workload (relins + rotations),
    from the circuit's structure: per query with C' = 2^r, 4 relinearisations
    per degree-9 polynomial, relins = 16 (r + 1) + r, rotations = r + 1
    (sign_dg = sign_df = 2)."""
    tot_relin, tot_rot = 0, 0
    for q in queries:
        r = (q.C - 1).bit_length()
        tot_relin += 16 * (r + 1) + r
        tot_rot += r + 1
    return tot_relin / len(queries), tot_rot / len(queries)


def run_reference(args, world, rank):
    from oracle import PRESETS
    from paper_2502_00847_gb300 import workloads
    if rank != 0:
        return
    P = PRESETS[args.params]
    qs = workloads.argmax_queries(args.queries, seed=4)
    relin_pq, rot_pq = op_mix_per_query(qs)
    times = []
    for i in range(args.warmup + args.steps):
        t_mul, t_rot, _, cores = oracle_sample(args.params, seconds_budget=5.0)
        per_query = relin_pq * t_mul + rot_pq * t_rot
        if i >= args.warmup:
            times.append(per_query)
    per_query = sum(times) / len(times)
    value = cores / per_query
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_query * 1e3 * args.queries,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batched encrypted ensemble Argmax, N=2^16, %d queries, K~U{4,8,16}, "
                               "C~U{2,3,4,6,14,64}" % args.queries, "queries": args.queries,
                   "params": "q0 60-bit + 23x50-bit, %d special 60-bit, dnum=%d, Delta=2^50" % (P.n_p, P.dnum)},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: oracle HMult+relin+rescale at levels 23/15/7 and one rotation "
                                   "at level 12, N=2^16, one copy per host core (%d, concurrent); queries/s = "
                                   "cores / per-query time extrapolated with the mix's %.1f relins + %.1f "
                                   "rotations per query" % (cores, relin_pq, rot_pq)},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- ours
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2502_00847_gb300.presets import PRESETS
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe, workloads

    pkg_build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    P = PRESETS[args.params]
    ctx = secpe.Context.from_params(P)
    keys = secpe.Keys(ctx, 1000 + rank, ROT_STEPS)
    n, cap = ctx.n, ctx.L + 1
    ct_words = 2 * cap * n

    c_choices = tuple(int(c) for c in args.classes.split(","))
    qs = rank_queries(args.queries, rank, c_choices)
    n_cts = sum(q.K for q in qs)
    # inputs: one big device tensor of ciphertexts, encrypted on the device
    inputs = torch.empty((n_cts, 2, cap, n), dtype=torch.int64, device=dev)
    views, off = [], 0
    for q in qs:
        cts = []
        for i in range(q.K):
            c = secpe.Ciphertext(inputs[off], 0, ctx.scale)
            secpe.encrypt_logits(ctx, keys, q.logits[i], q.d_min, q.enc_seeds[i], out=c)
            cts.append(c)
            off += 1
        views.append(cts)
    zbuf = torch.zeros((len(qs), 2, cap, n), dtype=torch.int64, device=dev)
    batch = [dict(cts=views[i], C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed,
                  z_out=secpe.Ciphertext(zbuf[i], 0, ctx.scale)) for i, q in enumerate(qs)]
    torch.cuda.synchronize()

    def step():
        secpe.argmax_batch(ctx, keys, batch)

    # launch configurations of the N = 2^16 kernels picked by the autotuner
    tuning = ctx.autotune()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness guard on the warm-up output: every query's index
    for i in range(len(qs)):
        zd = secpe.decrypt(ctx, keys, batch[i]["z_out"], qs[i].C)
        assert int(np.argmax(zd)) == int(np.argmax(qs[i].logits.mean(0))), "wrong argmax (query %d)" % i

    # the timed step: the whole batch as one captured CUDA graph (the
    # kernel-class events of the roofline are part of the graph and hold the
    # last replay's times), or the direct call
    graph = None
    timed_step = step
    if not args.no_graph:
        ctx.kprof_begin(args.kprof)
        graph = secpe.Graph(ctx, keys, batch)
        graph.launch()
        torch.cuda.synchronize()
        timed_step = graph.launch
    clocks = ClockSampler(local)
    ctx.reset_counters()
    if graph is None:
        ctx.kprof_begin(args.kprof)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        timed_step()
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    kp = ctx.kprof_end()
    kp_steps = 1 if graph is not None else args.steps
    graph_nodes = graph.nodes if graph is not None else None
    if graph is not None:
        graph.close()
        graph = None
    cnt = ctx.counters()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(world, ms)
    ms_per_step = ms / args.steps
    value = world * len(qs) * args.steps / (ms / 1e3)

    # per-kernel breakdown of one extra step (not part of the timed region)
    breakdown = None
    if args.breakdown:
        ctx.kprof_begin("*", max_launches=1 << 20)
        bev0, bev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        bev0.record()
        step()
        bev1.record()
        ctx.kprof_end()
        step_ms = bev0.elapsed_time(bev1)
        rows = ctx.kprof_report()
        breakdown = {"step_ms": step_ms, "kernel_ms": sum(r[2] for r in rows),
                     "kernels": [{"kernel": r[0], "launches": r[1], "ms": r[2], "share": r[2] / step_ms}
                                 for r in rows]}

    # the test-only refresh stand-in's share of one more (untimed) step, so
    # that the throughput without it can be stated too
    ctx.kprof_begin("refresh")
    rev0, rev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rev0.record()
    step()
    rev1.record()
    rkp = ctx.kprof_end()
    r_step_ms = rev0.elapsed_time(rev1)
    refresh = {"ms_per_step": rkp["total_ms"], "share": rkp["total_ms"] / r_step_ms,
               "refreshes_per_step": cnt["refreshes"] / args.steps,
               "value_excluding": len(qs) / ((r_step_ms - rkp["total_ms"]) / 1e3) * world,
               "note": "refresh = test-only stand-in for bootstrapping (decrypt, CRT lift, re-encrypt); "
                       "measured on one direct step after the timed region"}

    # plain path: the same kernels, one query per call, sequentially
    plain = None
    if args.plain_queries > 0 and rank == 0:
        npq = min(args.plain_queries, len(qs))
        # a sample of the mix with the same class-count distribution as the full mix
        idx = list(range(npq))
        zt = ctx.new_ct()
        for i in idx[:2]:
            y = secpe.ensemble_aggregate(ctx, batch[i]["cts"], qs[i].d_min, qs[i].d_max)
            secpe.encrypted_argmax(ctx, keys, y, qs[i].C, qs[i].qseed, out=zt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in idx:
            y = secpe.ensemble_aggregate(ctx, batch[i]["cts"], qs[i].d_min, qs[i].d_max)
            secpe.encrypted_argmax(ctx, keys, y, qs[i].C, qs[i].qseed, out=zt)
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": npq / (pms / 1e3), "unit": "queries/s", "queries": npq,
                 "note": "one ciphertext batch of 1 per launch, sequential; first %d queries of the mix" % npq}

    # end to end through host buffers (pinned): every step copies its inputs in
    # as seeded ciphertexts (c0 + the 8-byte encryption seed; c1 is regenerated
    # on the device by secpe_expand_seeded) and reads every z back.  Two input
    # sets alternate, so step s+1's host-to-device copy (on a copy stream) runs
    # under step s's evaluation; z is compacted on the device to the limbs of
    # its level and read back contiguously on the copy stream.
    e2e = None
    if not args.no_e2e:
        try:
            seeds = np.array([s_ for q in qs for s_ in q.enc_seeds], dtype=np.uint64)
            lv = max(b["z_out"].level for b in batch)
            host_c0 = torch.empty((n_cts, cap, n), dtype=torch.int64, pin_memory=True)
            host_c0.copy_(inputs[:, 0])
            inputs2 = torch.empty_like(inputs)
            zbuf2 = torch.zeros_like(zbuf)
            batch2, off = [], 0
            for i, q in enumerate(qs):
                cts = [secpe.Ciphertext(inputs2[off + k], c_.level, c_.scale) for k, c_ in enumerate(batch[i]["cts"])]
                off += q.K
                batch2.append(dict(batch[i], cts=cts, z_out=secpe.Ciphertext(zbuf2[i], 0, ctx.scale)))
            sets = [(inputs, batch, zbuf), (inputs2, batch2, zbuf2)]
            zc = [torch.empty((len(qs), 2, lv + 1, n), dtype=torch.int64, device=dev) for _ in range(2)]
            host_z = [torch.empty((len(qs), 2, lv + 1, n), dtype=torch.int64, pin_memory=True) for _ in range(2)]
            cs = torch.cuda.Stream()
            main = torch.cuda.current_stream()
            ev_in = [torch.cuda.Event() for _ in range(2)]
            ev_done = [torch.cuda.Event() for _ in range(2)]
            ev_free = [None, None]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier(world)
            e0.record()
            cs.wait_stream(main)

            def h2d(b):
                with torch.cuda.stream(cs):
                    if ev_free[b] is not None:
                        cs.wait_event(ev_free[b])
                    sets[b][0][:, 0].copy_(host_c0, non_blocking=True)
                    ev_in[b].record(cs)

            h2d(0)
            for s_ in range(args.steps):
                b = s_ % 2
                if s_ + 1 < args.steps:
                    h2d((s_ + 1) % 2)
                main.wait_event(ev_in[b])
                secpe.expand_seeded(ctx, sets[b][0], ctx.L, seeds)
                secpe.argmax_batch(ctx, keys, sets[b][1])
                zc[b].copy_(sets[b][2][:, :, : lv + 1])
                ev_done[b].record(main)
                with torch.cuda.stream(cs):
                    cs.wait_event(ev_done[b])
                    host_z[b].copy_(zc[b], non_blocking=True)
                    ev_free[b] = torch.cuda.Event()
                    ev_free[b].record(cs)
            main.wait_stream(cs)
            e1.record()
            torch.cuda.synchronize()
            ems = max_over_ranks(world, e0.elapsed_time(e1))
            # the read-back decrypts to the device result
            zq = secpe.Ciphertext(host_z[(args.steps - 1) % 2][0].cuda(), lv, batch[0]["z_out"].scale)
            zd = secpe.decrypt(ctx, keys, zq, qs[0].C)
            assert int(np.argmax(zd)) == int(np.argmax(qs[0].logits.mean(0))), "wrong argmax after read-back"
            e2e = {"value": world * len(qs) * args.steps / (ems / 1e3), "unit": "queries/s",
                   "h2d_bytes_per_step": int(n_cts * cap * n * 8 + seeds.nbytes),
                   "d2h_bytes_per_step": int(host_z[0].numel() * 8),
                   "transfer": "seeded ciphertexts: c0 + encryption seed host-to-device, c1 regenerated on "
                               "device; z read back at its level; two input sets, copies on a second stream "
                               "overlap the previous step"}
            del host_c0, host_z, inputs2, zbuf2, zc, batch2, sets
        except RuntimeError as e:
            e2e = {"value": None, "unit": "queries/s", "error": str(e)[:200]}

    cpu = None
    if not args.no_cpu and rank == 0:
        t_mul, t_rot, wall, cores = oracle_sample(args.params)
        relin_pq, rot_pq = op_mix_per_query(qs)
        per_query = relin_pq * t_mul + rot_pq * t_rot
        cpu = {"value": cores / per_query, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": "oracle HMult+relin+rescale at levels 23/15/7 and one rotation at level 12, N=2^16, "
                         "one copy per host core (%d, concurrent, %.1f s wall); one query per core, per-query "
                         "time extrapolated with the mix's %.1f relins + %.1f rotations"
                         % (cores, wall, relin_pq, rot_pq)}

    peak, peak_kind = hbm_peak()
    achieved = kp["bytes"] / (kp["total_ms"] / 1e3) / 1e9 if kp["total_ms"] > 0 else None
    roofline = {"bound": "hbm", "kernel": args.kprof, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                "traffic": (NTT16_DRAM_PER_ALG_BYTE * kp["bytes"] / max(1, kp["launches"])
                            if args.kprof == "ntt16" else None),
                "traffic_source": ("ncu DRAM bytes per algorithmic byte of the family in one HMult+relin+rescale "
                                   "of 8 ciphertexts (0.925), times this step's algorithmic bytes per launch"
                                   if args.kprof == "ntt16" else None),
                "launches_per_step": kp["launches"] / kp_steps,
                "kernel_ms_per_step": kp["total_ms"] / kp_steps,
                "bytes_per_launch": kp["bytes"] / max(1, kp["launches"])}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched encrypted ensemble Argmax, N=2^16, %d queries per GPU, "
                                   "K~U{4,8,16}, C~U{2,3,4,6,14,64}, seed 4" % len(qs),
                       "queries_per_gpu": len(qs), "input_ciphertexts": n_cts,
                       "params": "q0 60-bit + 23x50-bit, %d special 60-bit, dnum=%d, Delta=2^50" % (P.n_p, P.dnum),
                       "l2": "inputs (%.1f GB) larger than L2" % (n_cts * ct_words * 8 / 1e9),
                       "parallelism": "dp%d (independent queries per GPU)" % world,
                       "launch": ("one CUDA graph per step (%d nodes)" % graph_nodes) if graph_nodes
                                 else "direct call per step",
                       "autotune": {k: v["ctas_per_sm"] for k, v in tuning.items()}},
            "plain": plain, "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk, "gpu_launches": cnt["launches"], "refresh": refresh,
            **({"breakdown": breakdown} if breakdown else {}),
            "per_step_ops": {k: cnt[k] / args.steps for k in ("rotations", "signs", "relins", "refreshes",
                                                               "keyswitches")},
        }
        print(json.dumps(line))


def run_micro(args, rank):
    """Config-2 primitives on random residues (seed 2): batched NTT/INTT,
    key switching (algorithmic bytes = inputs + key + outputs), HMult +
    relinearise + rescale, rescale, rotation by 2^j (j = 0..15)."""
    import numpy as np
    import torch

    from paper_2502_00847_gb300.presets import PRESETS
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe

    pkg_build.build()
    ops = args.micro_ops.split(",")
    batches = [int(b) for b in args.micro_batch.split(",")]
    P = PRESETS[args.micro_params]
    ctx = secpe.Context.from_params(P)
    ctx.autotune()
    rot = [1 << j for j in range(16)] if "rotate" in ops else []
    keys = secpe.Keys(ctx, 2, rot)
    n, cap, L = ctx.n, ctx.L + 1, ctx.L
    primes = ctx.primes()
    gen = torch.Generator(device="cpu").manual_seed(2)
    limb = n * 8
    dnum = -(-ctx.n_q // -(-ctx.n_q // P.dnum))
    ksk_bytes = dnum * 2 * (cap + ctx.n_p) * limb

    def rand_batch(B):
        t = torch.empty((B, 2, cap, n), dtype=torch.int64)
        for i in range(cap):
            t[:, :, i] = torch.randint(0, primes[i], (B, 2, n), generator=gen, dtype=torch.int64)
        return t.cuda()

    def timed(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    res = {}
    for B in batches:
        x = rand_batch(B)
        y = rand_batch(B)
        out = torch.zeros_like(x)
        if "ntt" in ops:
            ms = timed(lambda: secpe.ntt_cts(ctx, x, B, 2 * cap * n, cap, L))
            res["ntt_B%d" % B] = {"ms": ms, "us_per_limb": ms * 1e3 / (B * 2 * cap),
                                  "GBps_alg": B * 2 * cap * limb * 4 / (ms / 1e3) / 1e9}
            ms = timed(lambda: secpe.ntt_cts(ctx, x, B, 2 * cap * n, cap, L, inverse=True))
            res["intt_B%d" % B] = {"ms": ms, "us_per_limb": ms * 1e3 / (B * 2 * cap)}
        a = secpe.CtBatch(x, L, ctx.scale)
        b = secpe.CtBatch(y, L, ctx.scale)
        o = secpe.CtBatch(out, 0, ctx.scale)
        if "ntt_tc" in ops:
            ms = timed(lambda: secpe.ntt_cts_tc(ctx, x, B, 2 * cap * n, cap, L))
            res["ntt_tc_B%d" % B] = {"ms": ms, "us_per_limb": ms * 1e3 / (B * 2 * cap),
                                     "GBps_alg": B * 2 * cap * limb * 4 / (ms / 1e3) / 1e9}
        if "ksk_tc" in ops:
            ms = timed(lambda: secpe.keyswitch_batch_tc(ctx, keys, 0, a, o))
            alg = B * (cap * limb + 2 * cap * limb) + ksk_bytes
            res["keyswitch_tc_B%d" % B] = {"ms": ms, "GBps_alg": alg / (ms / 1e3) / 1e9, "alg_bytes": alg}
        if "keyswitch" in ops:
            ms = timed(lambda: secpe.keyswitch_batch(ctx, keys, 0, a, o))
            alg = B * (cap * limb + 2 * cap * limb) + ksk_bytes
            res["keyswitch_B%d" % B] = {"ms": ms, "GBps_alg": alg / (ms / 1e3) / 1e9, "alg_bytes": alg}
        if "hmult" in ops:
            ms = timed(lambda: secpe.mul_relin_batch(ctx, keys, a, b, o))
            res["hmult_relin_rescale_B%d" % B] = {"ms": ms, "us_per_ct": ms * 1e3 / B}
        if "rescale" in ops:
            ms = timed(lambda: secpe.rescale_batch(ctx, a, o))
            res["rescale_B%d" % B] = {"ms": ms, "us_per_ct": ms * 1e3 / B}
        if args.micro_probe:
            probe = {"hmult": lambda: secpe.mul_relin_batch(ctx, keys, a, b, o),
                     "keyswitch": lambda: secpe.keyswitch_batch(ctx, keys, 0, a, o),
                     "ntt": lambda: secpe.ntt_cts(ctx, x, B, 2 * cap * n, cap, L)}[args.micro_probe]
            torch.cuda.synchronize()
            ctx.kprof_begin(args.kprof)
            torch.cuda.nvtx.range_push("micro_probe")
            probe()
            torch.cuda.nvtx.range_pop()
            kp = ctx.kprof_end()
            res["probe_%s_B%d" % (args.micro_probe, B)] = {"kprof": args.kprof, "launches": kp["launches"],
                                                           "alg_bytes": kp["bytes"], "ms": kp["total_ms"]}
        if "rotate" in ops:
            per = []
            for j in range(16):
                per.append(timed(lambda: secpe.rotate_batch(ctx, keys, a, 1 << j, o)))
            res["rotate_B%d" % B] = {"ms_mean": sum(per) / len(per), "ms_by_log2_step": per}
        del x, y, out
        torch.cuda.empty_cache()
    if "ntt_tc_identity" in ops:
        # precision variant: bit identity with the CUDA-core NTT over 10^4 seeded random ciphertexts
        total, chunk, mism = args.tc_identity_count, 50, 0
        t_tc = t_cc = 0.0
        for s0 in range(0, total, chunk):
            g2 = torch.Generator(device="cpu").manual_seed(30000 + s0)
            t = torch.empty((chunk, 2, cap, n), dtype=torch.int64)
            for i in range(cap):
                t[:, :, i] = torch.randint(0, primes[i], (chunk, 2, n), generator=g2, dtype=torch.int64)
            u = t.cuda()
            v = u.clone()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            secpe.ntt_cts(ctx, u, chunk, 2 * cap * n, cap, L)
            e[1].record()
            secpe.ntt_cts_tc(ctx, v, chunk, 2 * cap * n, cap, L)
            e[2].record()
            torch.cuda.synchronize()
            t_cc += e[0].elapsed_time(e[1])
            t_tc += e[1].elapsed_time(e[2])
            mism += int((u != v).any(dim=(1, 2, 3)).sum().item())
            secpe.ntt_cts(ctx, u, chunk, 2 * cap * n, cap, L, inverse=True)
            secpe.ntt_cts_tc(ctx, v, chunk, 2 * cap * n, cap, L, inverse=True)
            torch.cuda.synchronize()
            mism += int((u != v).any(dim=(1, 2, 3)).sum().item())
        res["ntt_tc_identity"] = {"ciphertexts": total, "mismatching_ciphertexts": mism,
                                  "forward_ms_cuda_cores": t_cc, "forward_ms_tensor_pipe": t_tc}
    if "ksk_tc_identity" in ops:
        # precision variant: key switching with tensor-pipe transforms and inner product, bit identity with
        # the CUDA-core key switch over seeded random ciphertexts (polynomial 0 of each, top level)
        total, chunk, mism = args.tc_identity_count, 50, 0
        t_tc = t_cc = 0.0
        for s0 in range(0, total, chunk):
            c = min(chunk, total - s0)
            g2 = torch.Generator(device="cpu").manual_seed(40000 + s0)
            t = torch.empty((c, 2, cap, n), dtype=torch.int64)
            for i in range(cap):
                t[:, :, i] = torch.randint(0, primes[i], (c, 2, n), generator=g2, dtype=torch.int64)
            dd = secpe.CtBatch(t.cuda(), L, ctx.scale)
            u = secpe.CtBatch(torch.zeros_like(dd.data), 0, ctx.scale)
            v = secpe.CtBatch(torch.zeros_like(dd.data), 0, ctx.scale)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            secpe.keyswitch_batch(ctx, keys, 0, dd, u)
            e[1].record()
            secpe.keyswitch_batch_tc(ctx, keys, 0, dd, v)
            e[2].record()
            torch.cuda.synchronize()
            t_cc += e[0].elapsed_time(e[1])
            t_tc += e[1].elapsed_time(e[2])
            mism += int((u.data != v.data).any(dim=(1, 2, 3)).sum().item())
            del dd, u, v
        res["ksk_tc_identity"] = {"ciphertexts": total, "mismatching_ciphertexts": mism, "level": L,
                                  "ms_cuda_cores": t_cc, "ms_tensor_pipe": t_tc}
    if rank == 0:
        desc = ("24x50-bit + 4x60-bit special primes, dnum=3" if args.micro_params == "micro" else
                "q0 60-bit + 23x50-bit + %dx60-bit special primes, dnum=%d" % (P.n_p, P.dnum))
        print(json.dumps({"mode": "micro", "config": {"workload": "primitive micro-benchmark N=2^16, %s, random "
                                                                  "residues seed 2" % desc},
                          "steps": args.steps, "warmup": args.warmup, "results": res}))


def run_serve(args, rank):
    """Serving loop (Poisson arrivals at each rate, continuous batching by
    secpe_server_*, admission by an HBM budget) against the plain path: the
    same queries served one at a time in arrival order (FIFO queue with the
    measured one-query service times)."""
    import numpy as np
    import torch

    from paper_2502_00847_gb300.presets import PRESETS
    from paper_2502_00847_gb300 import build as pkg_build
    from paper_2502_00847_gb300 import secpe, workloads

    pkg_build.build()
    ctx = secpe.Context.from_params(PRESETS[args.params])
    ctx.autotune()
    # one key set per tenant; pool query i belongs to tenant i % tenants
    tenants = [secpe.Keys(ctx, 1000 + rank + 7919 * t, ROT_STEPS) for t in range(args.tenants)]
    n, cap = ctx.n, ctx.L + 1
    pool = workloads.argmax_queries(64, seed=5)
    tkeys = [tenants[i % args.tenants] for i in range(len(pool))]
    n_cts = sum(q.K for q in pool)
    inputs = torch.empty((n_cts, 2, cap, n), dtype=torch.int64, device="cuda")
    views, off = [], 0
    for qi, q in enumerate(pool):
        cts = []
        for i in range(q.K):
            c = secpe.Ciphertext(inputs[off], 0, ctx.scale)
            secpe.encrypt_logits(ctx, tkeys[qi], q.logits[i], q.d_min, q.enc_seeds[i], out=c)
            cts.append(c)
            off += 1
        views.append(cts)
    # plain service time per pool query (one query per call)
    zt = ctx.new_ct()
    svc = []
    for i, q in enumerate(pool):
        torch.cuda.synchronize()
        t = time.perf_counter()
        y = secpe.ensemble_aggregate(ctx, views[i], q.d_min, q.d_max)
        secpe.encrypted_argmax(ctx, tkeys[i], y, q.C, q.qseed, out=zt)
        torch.cuda.synchronize()
        svc.append(time.perf_counter() - t)
    results = []
    rng = np.random.default_rng(5)
    for lam in [float(x) for x in args.rates.split(",")]:
        nq = args.serve_queries
        arrivals = np.cumsum(rng.exponential(1.0 / lam, nq))
        pick = rng.integers(0, len(pool), nq)
        srv = secpe.Server(ctx, tenants[0], hbm_budget_bytes=int(args.budget_gb * 1e9), max_batch=64)
        zbufs = {}
        pending = {}
        lat = []
        t0 = time.perf_counter()
        nxt = 0
        batch_sizes = []
        inflight = []  # one event per enqueued phase: bounds how far the host runs ahead of the GPU
        while nxt < nq or pending:
            now = time.perf_counter() - t0
            while nxt < nq and arrivals[nxt] <= now:
                i = int(pick[nxt])
                z = ctx.new_ct()
                tk = srv.submit(views[i], pool[i].C, pool[i].d_min, pool[i].d_max, pool[i].qseed + nxt, z,
                                keys=tkeys[i])
                pending[tk] = arrivals[nxt]
                zbufs[tk] = z
                nxt += 1
            launched = srv.step()
            if launched:
                batch_sizes.append(launched)
                ev = torch.cuda.Event()
                ev.record()
                inflight.append(ev)
                if len(inflight) > 4:
                    inflight.pop(0).synchronize()
            done = [tk for tk in pending if srv.poll(tk) == 1]
            now = time.perf_counter() - t0
            for tk in done:
                lat.append(now - pending.pop(tk))
                srv.forget(tk)
                zbufs.pop(tk)
            if not launched and not done and nxt < nq:
                time.sleep(max(0.0, min(0.002, arrivals[nxt] - now)))
            elif not launched and not done:
                torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        srv.close()
        # plain path: FIFO single server with the measured service times
        finish, plat = 0.0, []
        for a, i in zip(arrivals, pick):
            finish = max(finish, a) + svc[int(i)]
            plat.append(finish - a)
        lat = np.array(lat)
        plat = np.array(plat)
        results.append({"rate_qps": lam, "queries": nq,
                        "served": {"throughput_qps": nq / (wall - arrivals[0]), "p50_ms": 1e3 * np.median(lat),
                                   "p99_ms": 1e3 * np.percentile(lat, 99),
                                   "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0},
                        "plain": {"throughput_qps": nq / (finish - arrivals[0]), "p50_ms": 1e3 * np.median(plat),
                                  "p99_ms": 1e3 * np.percentile(plat, 99)}})
    if rank == 0:
        print(json.dumps({"mode": "serve", "metric": METRIC,
                          "config": {"workload": "serving loop: Poisson arrivals, %d queries per rate from a pool of "
                                                 "64 (K~U{4,8,16}, C~U{2,3,4,6,14,64}, seed 5), N=2^16, HBM "
                                                 "budget %.0f GB, max batch 64, %d tenant key set(s) resident"
                                                 % (args.serve_queries, args.budget_gb, args.tenants),
                                     "tenants": args.tenants},
                          "plain_service_ms_mean": 1e3 * float(np.mean(svc)), "rates": results}))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.serve:
        run_serve(args, rank)
    elif args.micro:
        run_micro(args, rank)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
