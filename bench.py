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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted ensemble-Argmax/s at N=2^16, batched vs plain; keyswitch GB/s; p99"
# DRAM bytes per byte that the launches themselves read and write (every
# transform pass a read and a write of each residue) of the N = 2^16
# transform-pass family (plain NTT/INTT passes, base-conversion pass A,
# inner-product and epilogue passes B), measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) over every family launch of
# one HMult + relinearise + rescale of 8 ciphertexts at level 23 (q0 + 23 x
# 50-bit, 8 special primes, dnum = 3): 2.831 GB of DRAM traffic against
# 3.045 GB read and written.  The step's family launches are the same
# kernels on more items, so their traffic is taken in the same proportion.
NTT16_DRAM_PER_MODEL_BYTE = 2.831 / 3.045
# integer multiply pipe: 152 SMs, 64 32-bit multiplies (IMAD-class) per clock per SM
SM_COUNT = 152
MUL32_PER_CLK_PER_SM = 64
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
    ap.add_argument("--plain-queries", type=int, default=-1,
                    help="queries timed on the one-query-per-launch path (-1: all of the mix, 0: none)")
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
    ap.add_argument("--micro-ops", default="ntt,keyswitch,hmult,rescale,rotate",
                    help="also: ntt_tc, ksk_tc, ntt_tc_identity, word32 (the word-size probe)")
    ap.add_argument("--micro-batch", default="1,8,64")
    ap.add_argument("--micro-probe", default="", choices=["", "hmult", "keyswitch", "ntt"],
                    help="after timing, one more call of this op inside the NVTX range 'micro_probe' with the "
                         "--kprof class profiled (its algorithmic bytes, for DRAM-traffic captures)")
    ap.add_argument("--tc-identity-count", type=int, default=10000,
                    help="seeded random ciphertexts of the precision variant's bit-identity checks")
    ap.add_argument("--serve", action="store_true",
                    help="serving loop: Poisson arrivals, continuous batching, p50/p99 latency")
    ap.add_argument("--rates", default="50,200,500,1000,2000")
    ap.add_argument("--serve-rate", type=float, default=64.0,
                    help="default run: one short serving run at this rate (queries/s; 0: none)")
    ap.add_argument("--serve-window", type=float, default=8.0, help="default run: its arrival window (s)")
    ap.add_argument("--no-boot", dest="boot", action="store_false",
                    help="default run: skip the bootstrapping leg")
    ap.add_argument("--ni-queries", type=int, default=64,
                    help="default run: queries of the non-interactive (bootstrapped) Argmax leg (0: none)")
    ap.add_argument("--no-clip", dest="clip", action="store_false",
                    help="default run: skip the CLIP-style linear-step pipeline")
    ap.add_argument("--no-phoenix", dest="phoenix", action="store_false",
                    help="default run: skip the Phoenix baseline legs")
    ap.add_argument("--packed-sets", type=int, default=256,
                    help="default run: packed query sets of the slot-packing line (0: none)")
    ap.add_argument("--no-keyswitch-gbps", dest="keyswitch_gbps", action="store_false",
                    help="default run: skip the primitive-set key-switch GB/s")
    ap.add_argument("--no-word32", dest="word32", action="store_false",
                    help="skip the word-size probe (32-bit against 64-bit residues)")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="arrival window per rate")
    ap.add_argument("--serve-queries", type=int, default=3000, help="at most this many queries per rate")
    ap.add_argument("--no-plain-serve", action="store_true", help="serving: skip the plain path's real run")
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
# The CPU oracle (test infrastructure) is run only by the cpu_baseline leg of
# the GPU arm and by the reference arm, in worker processes started with
# spawn.
ORACLE_KEY_SEED = 4711
ORACLE_ROT = (-2, 1)


def oracle_cores():
    return max(1, min(16, os.cpu_count() or 1))


def oracle_pool(cores):
    import multiprocessing
    return multiprocessing.get_context("spawn").Pool(cores)


def op_mix_per_query(queries):
    """Key switches per query of the workload, from the circuit's structure:
    with C' = 2^r, 4 relinearisations per degree-9 polynomial, 16 per Sign,
    r + 1 Signs and r products of Max: relins = 16 (r + 1) + r; rotations =
    r + 1 (sign_dg = sign_df = 2).  The GPU counters of a step equal these."""
    tot_relin, tot_rot = 0, 0
    for q in queries:
        r = (q.C - 1).bit_length()
        tot_relin += 16 * (r + 1) + r
        tot_rot += r + 1
    return tot_relin / len(queries), tot_rot / len(queries)


def oracle_whole_queries(pool, cores, params_name):
    """Every host core runs one whole query (C = 2, K = 4: ensemble
    aggregation + Alg. 1 at N = 2^16, the cheapest query of the mix)
    concurrently; returns its mean time, key switches and refreshes."""
    from oracle import jobs as ojobs
    from paper_2502_00847_gb300 import workloads
    qs = [workloads.argmax_queries(1, seed=500 + i, K_choices=(4,), C_choices=(2,))[0] for i in range(cores)]
    jobs = [(params_name, ORACLE_KEY_SEED, ORACLE_ROT, q.logits, q.d_min, q.d_max, q.qseed, q.enc_seeds)
            for q in qs]
    t0 = time.perf_counter()
    res = pool.map(ojobs.ensemble_query, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    for q, r in zip(qs, res):
        assert int(np.argmax(r["decoded"])) == int(np.argmax(q.logits.mean(0))), "oracle argmax wrong"
    c = res[0]["counters"]
    return {"t_query": statistics.mean(r["seconds"] for r in res),
            "ks_query": c["relins"] + c["rotations"], "refreshes": c["refreshes"], "wall": wall}


def cpu_rate(whole, ks_mix):
    """queries/s of the host cores on the mix: the measured whole query's time
    per key switch times the mix's key switches per query."""
    return whole["cores"] * whole["ks_query"] / (ks_mix * whole["t_query"])


def cpu_baseline_line(whole, ks_mix, relin_pq, rot_pq, value=None):
    v = cpu_rate(whole, ks_mix) if value is None else value
    return {"value": v, "unit": "queries/s", "cores": whole["cores"], "kind": "oracle",
            "sample": "each of %d host cores ran one whole query of the workload (C=2, K=4: aggregation + "
                      "Alg. 1 at N=2^16, %d key switches, %d refresh) concurrently: %.1f s per query; scaled to "
                      "the mix by key switches per query (%.1f relins + %.1f rotations); %.0f s wall"
                      % (whole["cores"], whole["ks_query"], whole["refreshes"], whole["t_query"], relin_pq,
                         rot_pq, whole["wall"])}


def workloads_argmax_queries(n):
    from paper_2502_00847_gb300 import workloads
    return workloads.argmax_queries(n, seed=4)


def run_reference(args, world, rank):
    """The oracle as it stands on the host cores.  Before the steps, every core
    runs one whole query (the calibration above, untimed); each step then is
    a bounded sample of the workload: every core runs one HMult +
    relinearisation + rescale at one of 16 levels spread over 2..L (the
    circuit's dominant operation over the levels it visits), concurrently.
    A step's rate is the whole-query rate scaled by how fast that sample ran
    against the same sample in the first warm-up step."""
    from oracle import PRESETS
    from oracle import jobs as ojobs
    if rank != 0:
        return
    P = PRESETS[args.params]
    qs = workloads_argmax_queries(args.queries)
    relin_pq, rot_pq = op_mix_per_query(qs)
    ks_mix = relin_pq + rot_pq
    cores = oracle_cores()
    L = P.n_q - 1
    levels = [2 + round(i * (L - 2) / (cores - 1)) if cores > 1 else L for i in range(cores)]
    pool = oracle_pool(cores)
    try:
        whole = oracle_whole_queries(pool, cores, args.params)
        whole["cores"] = cores
        base_rate = cpu_rate(whole, ks_mix)
        ref_t, rates, walls = None, [], []
        for i in range(args.warmup + args.steps):
            jobs = [(args.params, ORACLE_KEY_SEED, ORACLE_ROT, lv, 1000 * i + c) for c, lv in enumerate(levels)]
            t0 = time.perf_counter()
            ts = pool.map(ojobs.hmult_sample, jobs, chunksize=1)
            wall = time.perf_counter() - t0
            t_mean = statistics.mean(ts)
            if ref_t is None:
                ref_t = t_mean
            if i >= args.warmup:
                rates.append(base_rate * ref_t / t_mean)
                walls.append(wall)
    finally:
        pool.close()
        pool.join()
    value = statistics.mean(rates)
    cb = cpu_baseline_line(whole, ks_mix, relin_pq, rot_pq, value=value)
    cb["sample"] += ("; per step: one HMult+relin+rescale per core at levels %s, concurrently (%.2f s wall per "
                     "step); a step's rate = the whole-query rate x (first warm-up sample time / step sample time)"
                     % (levels, statistics.mean(walls)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batched encrypted ensemble Argmax, N=2^16, %d queries, K~U{4,8,16}, "
                               "C~U{2,3,4,6,14,64}, seed 4" % args.queries, "queries": args.queries,
                   "params": "q0 60-bit + 23x50-bit, %d special 60-bit, dnum=%d, Delta=2^50" % (P.n_p, P.dnum)},
        "cpu_baseline": cb,
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
    torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler capture exactly these launches
    ev0.record()
    for _ in range(args.steps):
        timed_step()
    ev1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
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

    # plain path: the same kernels, one query per call, sequentially, over
    # every query of the mix (the same workload as the batched step)
    plain = None
    if args.plain_queries != 0 and rank == 0:
        npq = len(qs) if args.plain_queries < 0 else min(args.plain_queries, len(qs))
        zt = ctx.new_ct()
        for i in range(min(2, npq)):
            y = secpe.ensemble_aggregate(ctx, batch[i]["cts"], qs[i].d_min, qs[i].d_max)
            secpe.encrypted_argmax(ctx, keys, y, qs[i].C, qs[i].qseed, out=zt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(npq):
            y = secpe.ensemble_aggregate(ctx, batch[i]["cts"], qs[i].d_min, qs[i].d_max)
            secpe.encrypted_argmax(ctx, keys, y, qs[i].C, qs[i].qseed, out=zt)
        e1.record()
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": npq / (pms / 1e3), "unit": "queries/s", "queries": npq,
                 "note": "one query per call (aggregate + encrypted_argmax, batch of 1 per launch), sequential, "
                         "%s" % ("every query of the mix" if npq == len(qs) else "first %d queries" % npq)}

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

    # a short serving run at one rate (continuous batching vs the plain path,
    # both run for real on the same arrivals), on the resident mix
    serve = None
    if args.serve_rate > 0 and rank == 0:
        serve = serve_rate(ctx, keys, [keys] * len(qs), [b["cts"] for b in batch], qs, args.serve_rate,
                           args.serve_window, 5, int(args.budget_gb * 1e9), 64, 10 ** 6)

    # the Phoenix baseline (Sec. 3.2) on the same queries and GPU, and the
    # paper's comparison point n = 256
    phoenix = (run_phoenix(secpe, torch, workloads, ctx, batch, qs, 1000 + rank, ms_per_step)
               if args.phoenix and rank == 0 else None)

    # the CLIP-style pipeline: encrypted linear step (K = 80 templates) +
    # aggregation + Argmax for a batch of encrypted images
    clip = run_clip(secpe, torch, workloads, ctx, 1000 + rank) if args.clip and rank == 0 else None

    # key switching of the primitive set (config 2: 24 x 50-bit + 4 special,
    # dnum = 3) at B = 1 and B = 8, algorithmic bytes = input + key + output
    ksw = keyswitch_gbps(secpe, torch, dev, args.steps) if args.keyswitch_gbps and rank == 0 else None
    word = word_size_probe(secpe, torch, dev, args.steps) if args.word32 and rank == 0 else None

    # measured throughput of the integer multiply pipe (the ALU roofline)
    probe = ctx.mul32_probe() if rank == 0 else None

    # rooflines of the N = 2^16 transform-pass family (the kernel class timed
    # live over the timed step): HBM (algorithmic bytes) and integer ALU
    # (algorithmic 32-bit multiplies); the binding one is the higher fraction
    hbm, hbm_kind = hbm_peak()
    fam_s = kp["total_ms"] / 1e3
    per_launch = lambda x: x / max(1, kp["launches"])
    gbs = kp["bytes"] / fam_s / 1e9 if fam_s > 0 else None
    r_hbm = {"bound": "hbm", "kernel": args.kprof, "achieved": gbs, "peak": hbm, "unit": "GB/s",
             "frac": gbs / hbm if gbs else None, "peak_kind": hbm_kind,
             "traffic": (NTT16_DRAM_PER_MODEL_BYTE * per_launch(kp["model_bytes"]) if args.kprof == "ntt16" else None),
             "traffic_source": ("ncu dram bytes read+write per byte the family's launches read and write "
                                "(0.930, one HMult+relin+rescale of 8 ciphertexts), times this step's such bytes "
                                "per launch" if args.kprof == "ntt16" else None),
             "bytes_per_launch": per_launch(kp["bytes"]),
             "traffic_model": per_launch(kp["model_bytes"]),
             "traffic_model_note": "bytes each launch itself reads and writes (every transform pass a read and a "
                                   "write of each residue, intermediates included)"}
    smax = clk.get("sm_max_mhz") or 2070.0
    alu_peak = MUL32_PER_CLK_PER_SM * SM_COUNT * smax * 1e6 / 1e12
    tmul = kp["mul32"] / fam_s / 1e12 if fam_s > 0 else None
    r_alu = {"bound": "alu", "kernel": args.kprof, "achieved": tmul, "peak": alu_peak, "unit": "Tmul32/s",
             "frac": tmul / alu_peak if tmul else None,
             "peak_kind": "derived: %d SMs x %d 32-bit multiplies per clock per SM x %.0f MHz"
                          % (SM_COUNT, MUL32_PER_CLK_PER_SM, smax),
             "probe": probe / 1e12 if probe else None,
             "frac_of_probe": (tmul / (probe / 1e12)) if (tmul and probe) else None,
             "probe_note": "secpe_mul32_probe: 128-bit multiply-accumulate chains (8 32-bit multiplies each) "
                           "on register data, all SMs",
             "mul32_per_launch": per_launch(kp["mul32"]),
             # the same launches' DRAM traffic (a property of the kernels, whichever roofline binds)
             "traffic": r_hbm["traffic"], "traffic_source": r_hbm["traffic_source"]}
    common = {"launches_per_step": kp["launches"] / kp_steps, "kernel_ms_per_step": kp["total_ms"] / kp_steps,
              "family_share_of_step": (kp["total_ms"] / kp_steps) / ms_per_step}
    r_hbm.update(common)
    r_alu.update(common)
    roofline, other = (r_alu, r_hbm) if (r_alu["frac"] or 0) >= (r_hbm["frac"] or 0) else (r_hbm, r_alu)

    # free the device state of the one-query-per-ciphertext mix
    del inputs, zbuf, batch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # CKKS bootstrapping (the non-interactive replacement of the refresh
    # stand-in) at N = 2^16 on its own parameter set
    boot = run_boot(secpe, torch, dev, refresh) if args.boot and rank == 0 else None
    if boot is not None and args.ni_queries > 0:
        boot["noninteractive_argmax"] = run_noninteractive(secpe, torch, workloads, dev, args.ni_queries)

    # slot-packed multi-query Argmax: the mix's tasks, every ciphertext set
    # filled to capacity (N/(4C') inputs per ciphertext)
    packed = (run_packed(secpe, torch, workloads, ctx, keys, dev, min(args.steps, 5), args.packed_sets)
              if args.packed_sets and rank == 0 else None)

    cpu = None
    if not args.no_cpu and rank == 0:
        relin_pq, rot_pq = op_mix_per_query(qs)
        cores = oracle_cores()
        pool = oracle_pool(cores)
        try:
            whole = oracle_whole_queries(pool, cores, args.params)
        finally:
            pool.close()
            pool.join()
        whole["cores"] = cores
        cpu = cpu_baseline_line(whole, relin_pq + rot_pq, relin_pq, rot_pq)

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
                       "refresh": "test-only interactive stand-in for bootstrapping (decrypt, CRT lift, "
                                  "re-encrypt), included in every step",
                       "autotune": {k: v["ctas_per_sm"] for k, v in tuning.items()}},
            "plain": plain, "e2e": e2e, "roofline": roofline, "roofline_other": other, "cpu_baseline": cpu,
            "keyswitch_GBps": ksw, "word_size": word, "serve": serve, "packed": packed, "phoenix": phoenix, "clip": clip,
            "bootstrap": boot,
            "p99_ms": serve["served"]["p99_ms"] if serve else None,
            "clocks": clk, "gpu_launches": cnt["launches"], "refresh": refresh,
            **({"breakdown": breakdown} if breakdown else {}),
            "per_step_ops": {k: cnt[k] / args.steps for k in ("rotations", "signs", "relins", "refreshes",
                                                               "keyswitches")},
        }
        print(json.dumps(line))


def run_phoenix(secpe, torch, workloads, ctx, batch, qs, key_seed, secpe_ms):
    """The Phoenix Argmax (m = C' - 1 comparisons + 1 Sign) over the whole mix
    as one secpe_phoenix_argmax_batch call (one warm-up, one timed step),
    against the SecPE step; and one query with n = C = 256 (K = 4), SecPE's
    one-query call against Phoenix's, the paper's comparison point."""
    keys = secpe.Keys(ctx, key_seed, list(range(1, 64)) + [-2, -4, -8, -16, -64])
    pb = [dict(b, z_out=ctx.new_ct()) for b in batch]
    secpe.phoenix_argmax_batch(ctx, keys, pb)
    torch.cuda.synchronize()
    for q, b in zip(qs, pb):
        zd = secpe.decrypt(ctx, keys, b["z_out"], q.C)
        assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0))), "wrong Phoenix argmax"
    ctx.reset_counters()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    secpe.phoenix_argmax_batch(ctx, keys, pb)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cnt = ctx.counters()
    del pb
    keys.close()
    out = {"value": len(qs) / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
           "secpe_over_phoenix": ms / secpe_ms,
           "per_step_ops": {k: cnt[k] for k in ("signs", "rotations", "relins", "refreshes")},
           "workload": "the same 256-query mix, one secpe_phoenix_argmax_batch call per step (direct)"}
    # the paper's comparison point: one query of n = 256 classes
    k256 = secpe.Keys(ctx, key_seed + 1, list(range(1, 256)) + [-256])
    q = workloads.argmax_queries(1, seed=256, K_choices=(4,), C_choices=(256,))[0]
    cts = [secpe.encrypt_logits(ctx, k256, q.logits[i], q.d_min, q.enc_seeds[i]) for i in range(q.K)]
    y = secpe.ensemble_aggregate(ctx, cts, q.d_min, q.d_max)
    times = {}
    for name, fn in (("secpe", secpe.encrypted_argmax), ("phoenix", secpe.phoenix_argmax)):
        z = fn(ctx, k256, y, q.C, q.qseed)
        torch.cuda.synchronize()
        assert int(np.argmax(secpe.decrypt(ctx, k256, z, q.C))) == int(np.argmax(q.logits.mean(0))), name
        ctx.reset_counters()
        e0.record()
        fn(ctx, k256, y, q.C, q.qseed, out=z)
        e1.record()
        torch.cuda.synchronize()
        c = ctx.counters()
        times[name] = {"ms": e0.elapsed_time(e1), "signs": c["signs"], "rotations": c["rotations"],
                       "relins": c["relins"]}
    k256.close()
    out["n256"] = dict(times, speedup=times["phoenix"]["ms"] / times["secpe"]["ms"],
                       paper_speedup=20.8,
                       note="one query, n = C = 256, K = 4, each Argmax one call; the paper's 20.8x is SEAL+HEXL "
                            "on a CPU (Sec. 4.5), context only")
    return out


def run_clip(secpe, torch, workloads, ctx, key_seed, d=512, C=10, K=80, B=16):
    """CLIP-style prompt ensembling (Sec. 2.3) end to end on the device: one
    task's plaintext text embeddings T[K][C][d] (K = 80 templates), B
    encrypted image embeddings; per image secpe_linear_apply (K logit
    ciphertexts, batched over the prompts), then one secpe_argmax_batch over
    the B images.  One warm-up, one timed pass."""
    cp = 1 << (C - 1).bit_length()
    rot = [cp << t for t in range(d.bit_length() - 1)] + [-cp] + [1 << i for i in range(cp.bit_length() - 1)]
    keys = secpe.Keys(ctx, key_seed, rot)
    T, xs, qseeds, seeds = workloads.clip_images(d, C, K, B)
    lin = secpe.Linear(ctx, T=T, d_min=workloads.ARGMAX_BOUNDS[0])
    xcts = [secpe.encrypt_replicated(ctx, keys, x, C, s) for x, s in zip(xs, seeds)]
    outs = [[ctx.new_ct() for _ in range(K)] for _ in range(B)]
    batch = [dict(cts=outs[b], C=C, d_min=workloads.ARGMAX_BOUNDS[0], d_max=workloads.ARGMAX_BOUNDS[1],
                  qseed=qseeds[b], z_out=ctx.new_ct()) for b in range(B)]
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))

    def run():
        e0.record()
        for b in range(B):
            lin.apply(keys, xcts[b], outs[b])
        e1.record()
        secpe.argmax_batch(ctx, keys, batch)
        e2.record()
        torch.cuda.synchronize()

    run()
    for b in range(B):
        zd = secpe.decrypt(ctx, keys, batch[b]["z_out"], C)
        assert int(np.argmax(zd)) == int(np.argmax(np.einsum("kcd,d->kc", T, xs[b]).mean(0))), "wrong CLIP argmax"
    ctx.reset_counters()
    run()
    cnt = ctx.counters()
    ms_lin, ms_arg = e0.elapsed_time(e1), e1.elapsed_time(e2)
    lin.close()
    keys.close()
    del outs, batch, xcts
    return {"value": B / ((ms_lin + ms_arg) / 1e3), "unit": "images/s", "images": B, "ms_linear": ms_lin,
            "ms_argmax": ms_arg, "rotations": cnt["rotations"],
            "workload": "CLIP-style zero-shot: d=%d, C=%d, K=%d templates, %d encrypted images; per image the "
                        "linear step (K plaintext products, log2(d) rotate-adds batched over the prompts, mask, "
                        "pad), then aggregation + Alg. 1 for all images in one batch" % (d, C, K, B)}


def run_boot(secpe, torch, dev, refresh, n=128, batches=(1, 16)):
    """Sparse-slot CKKS bootstrapping (secpe_bootstrap_batch) at N = 2^16 on
    the boot16 set (q0 50-bit, 10 x 40-bit computation primes, 16 x 60-bit
    bootstrapping primes, 5 special, dnum 7, sparse secret h = 32), blocks of
    n = 128 slots (2C' for C' <= 64): one warm-up, then 3 timed batches at
    each batch size (inside the NVTX range "boot_B<size>"); checked against
    the input slots."""
    from paper_2502_00847_gb300.presets import BOOT16
    ctx = secpe.Context.from_params(BOOT16)
    ctx.autotune()
    keys = secpe.Keys(ctx, 77, secpe.boot_rotation_steps(ctx, n))
    t0 = time.perf_counter()
    bt = secpe.Boot(ctx, n)
    t_plan = time.perf_counter() - t0
    rng = np.random.default_rng(16)
    out = {"params": "boot16: N=2^16, q0 50-bit, 10x40-bit computation + 16x60-bit bootstrapping primes, "
                     "5 special 60-bit, dnum=7, sparse secret h=32", "block_slots": n,
           "levels_consumed": 16, "output_level": ctx.L - 16, "plan_s": t_plan}
    for B in batches:
        vs = rng.uniform(-1, 1, (B, n // 2))
        data = torch.zeros((B, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device=dev)
        for b in range(B):
            # n-periodic inputs (n/2 values and n/2 zeros in every block of n slots), which
            # bootstrapping returns unchanged
            secpe.encrypt_logits_packed(ctx, keys, np.tile(vs[b], (ctx.n // (2 * n), 1)), 0.0, 400 + b,
                                        out=secpe.Ciphertext(data[b], 0, ctx.scale))
        res = secpe.CtBatch(torch.zeros_like(data), 0, 0.0)
        x = secpe.CtBatch(data, 0, ctx.scale)
        bt.bootstrap_batch(keys, x, res)
        torch.cuda.synchronize()
        err = max(float(np.max(np.abs(secpe.decrypt(ctx, keys, secpe.Ciphertext(res.data[b], res.level, res.scale),
                                                     n // 2) - vs[b]))) for b in range(min(B, 4)))
        assert err < 2.0 ** -16, "bootstrap error %g" % err
        ctx.reset_counters()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("boot_B%d" % B)
        e0.record()
        for _ in range(3):
            bt.bootstrap_batch(keys, x, res)
        e1.record()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        cnt = ctx.counters()
        out["B%d" % B] = {"ms": ms, "ms_per_ciphertext": ms / B, "max_abs_error": err,
                          "rotations": cnt["rotations"] / 3 / B, "relins": cnt["relins"] / 3 / B}
        del data, res, x
    bt.close()
    keys.close()
    ctx.close()
    per = out["B%d" % batches[-1]]["ms_per_ciphertext"]
    out["refresh_stand_in_ms_per_ciphertext"] = refresh["ms_per_step"] / max(1.0, refresh["refreshes_per_step"])
    out["step_if_bootstrapped_ms_estimate"] = refresh["refreshes_per_step"] * per
    out["note"] = ("non-interactive; the Argmax parameter set has no bootstrapping primes, so the benchmark step "
                   "keeps the refresh stand-in; the estimate prices each of its refreshes at one batched bootstrap")
    return out


def run_noninteractive(secpe, torch, workloads, dev, n_queries, n=128, n_sets=16):
    """The whole encrypted ensemble Argmax without the interactive stand-in:
    queries of the mix (seed 4, the first n_queries) on boot16, each prompt's
    logits packed into every 2C'-block (inputs 2C'-periodic, at the top
    computation level L - 16), one secpe_argmax_batch_boot call with every
    refresh a batched bootstrap (block n = 128).  One warm-up on 4 queries,
    one timed call; every query's index checked.  Then slot-packed: n_sets
    sets of the mix's tasks with n / (2C') different inputs in every 128-slot
    block, one timed call, every input's index checked."""
    from paper_2502_00847_gb300.presets import BOOT16
    ctx = secpe.Context.from_params(BOOT16)
    ctx.autotune()
    keys = secpe.Keys(ctx, 78, sorted(set(secpe.boot_rotation_steps(ctx, n)) | set(ROT_STEPS)))
    bt = secpe.Boot(ctx, n)
    qs = workloads.argmax_queries(n_queries, seed=4)
    lv = ctx.L - 16
    n_cts = sum(q.K for q in qs)
    data = torch.empty((n_cts, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device=dev)
    batch, off = [], 0
    for q in qs:
        P = secpe.packed_capacity(16, q.C)
        cts = []
        for i in range(q.K):
            c = secpe.Ciphertext(data[off], 0, ctx.scale)
            secpe.encrypt_logits_packed(ctx, keys, np.tile(q.logits[i], (P, 1)), q.d_min, q.enc_seeds[i], out=c)
            c.level = lv
            cts.append(c)
            off += 1
        batch.append(dict(cts=cts, C=q.C, d_min=q.d_min, d_max=q.d_max, qseed=q.qseed, z_out=ctx.new_ct()))
    secpe.argmax_batch_boot(ctx, keys, bt, batch[:4])
    torch.cuda.synchronize()
    ctx.reset_counters()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    secpe.argmax_batch_boot(ctx, keys, bt, batch)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cnt = ctx.counters()
    ok = sum(int(np.argmax(secpe.decrypt(ctx, keys, b["z_out"], q.C))) == int(np.argmax(q.logits.mean(0)))
             for q, b in zip(qs, batch))
    del data, batch
    out = {"value": n_queries / (ms / 1e3), "unit": "queries/s", "queries": n_queries, "ms": ms,
           "bootstraps_per_query": cnt["bootstraps"] / n_queries, "relins_per_query": cnt["relins"] / n_queries,
           "correct_indices": ok,
           "workload": "the first %d queries of the mix on boot16 (Delta = 2^40, 10 computation levels between "
                       "bootstraps), inputs packed 2C'-periodic, every refresh a batched bootstrap" % n_queries}
    # slot-packed: n / (2C') different inputs of one task in every n-block
    # (the block repeated over the N/2 slots, so the bootstrap's n-periodic
    # average keeps it), one ciphertext per prompt for all of them
    sets = workloads.packed_queries(n_sets, n, seed=7)
    S = ctx.n // 2
    n_cts = sum(st.K for st in sets)
    data = torch.empty((n_cts, 2, ctx.L + 1, ctx.n), dtype=torch.int64, device=dev)
    batch, off = [], 0
    for st in sets:
        cts = []
        for i in range(st.K):
            c = secpe.Ciphertext(data[off], 0, ctx.scale)
            secpe.encrypt_logits_packed(ctx, keys, np.tile(st.prompt(i), (S // n, 1)), st.d_min, st.enc_seeds[i],
                                        out=c)
            c.level = lv
            cts.append(c)
            off += 1
        batch.append(dict(cts=cts, C=st.C, d_min=st.d_min, d_max=st.d_max, qseed=st.qseed, z_out=ctx.new_ct()))
    torch.cuda.synchronize()
    ctx.reset_counters()
    e0.record()
    secpe.argmax_batch_boot(ctx, keys, bt, batch)
    e1.record()
    torch.cuda.synchronize()
    msp = e0.elapsed_time(e1)
    cnt = ctx.counters()
    inputs = sum(st.P for st in sets)
    okp = 0
    for st, b in zip(sets, batch):
        cp = 1 << (st.C - 1).bit_length()
        z = secpe.decrypt_packed(ctx, keys, b["z_out"], S // (2 * cp), st.C)
        okp += sum(int(np.argmax(z[j])) == int(np.argmax(st.logits[j].mean(0))) for j in range(st.P))
    out["packed"] = {"value": inputs / (msp / 1e3), "unit": "queries/s", "inputs": inputs, "sets": n_sets,
                     "ms": msp, "bootstraps_per_set": cnt["bootstraps"] / n_sets, "correct_indices": okp,
                     "workload": "%d sets of the mix's tasks (seed 7), each n / (2C') inputs per 128-slot block "
                                 "(the block repeated over the slots), on boot16, every refresh a batched "
                                 "bootstrap" % n_sets}
    bt.close()
    keys.close()
    del data, batch
    ctx.close()
    return out


def run_packed(secpe, torch, workloads, ctx, keys, dev, steps, n_sets=256):
    """Slot packing (SecPE Sec. 3.2 after Alg. 1): n_sets packed query sets
    drawn like the mix's queries (K ~ U{4,8,16}, C ~ U{2,...,64}, seed 6),
    each filled to N/(4C') inputs, encrypted by the library's packed encoder;
    one step = secpe_argmax_batch over all sets (the same circuit as the
    one-query-per-ciphertext step, on full slot vectors)."""
    sets = workloads.packed_queries(n_sets, ctx.n // 2, seed=6)
    n_cts = sum(s.K for s in sets)
    cap = ctx.L + 1
    t0 = time.perf_counter()
    data = torch.empty((n_cts, 2, cap, ctx.n), dtype=torch.int64, device=dev)
    batch, off = [], 0
    for s in sets:
        cts = []
        for i in range(s.K):
            c = secpe.Ciphertext(data[off], 0, ctx.scale)
            secpe.encrypt_logits_packed(ctx, keys, s.prompt(i), s.d_min, s.enc_seeds[i], out=c)
            cts.append(c)
            off += 1
        batch.append(dict(cts=cts, C=s.C, d_min=s.d_min, d_max=s.d_max, qseed=s.qseed, z_out=ctx.new_ct()))
    torch.cuda.synchronize()
    t_enc = time.perf_counter() - t0
    secpe.argmax_batch(ctx, keys, batch)
    torch.cuda.synchronize()
    # every input of the first sets against its exact argmax
    checked = 0
    for s, b in list(zip(sets, batch))[:8]:
        zd = secpe.decrypt_packed(ctx, keys, b["z_out"], s.P, s.C)
        assert np.array_equal(zd.argmax(1), s.logits.mean(1).argmax(1)), "wrong packed argmax"
        checked += s.P
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        secpe.argmax_batch(ctx, keys, batch)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    inputs = sum(s.P for s in sets)
    del batch, data
    torch.cuda.empty_cache()
    return {"value": inputs / (ms / 1e3), "unit": "queries/s", "inputs_per_step": inputs, "sets": len(sets),
            "input_ciphertexts": n_cts, "ms_per_step": ms, "steps": steps, "inputs_checked": checked,
            "encrypt_s": t_enc,
            "workload": "slot-packed: %d query sets with the mix's K and C (seed 6), each filled to N/(4C') "
                        "inputs per ciphertext; one step = secpe_argmax_batch over all sets (direct call)"
                        % len(sets)}


def keyswitch_gbps(secpe, torch, dev, steps):
    """Key switching with the relinearisation key of the primitive set (N =
    2^16, 24 x 50-bit + 4 x 60-bit special primes, dnum = 3) on uniform
    residues (seed 2) at B = 1 and B = 8 items per launch; GB/s of
    algorithmic bytes (input B (L+1) limbs + key 2 dnum (L+1+k) limbs + output
    2 B (L+1) limbs, 8 N bytes each) over the mean launch time."""
    from paper_2502_00847_gb300.presets import MICRO
    ctx = secpe.Context.from_params(MICRO)
    ctx.autotune()
    keys = secpe.Keys(ctx, 2, [])
    n, cap, L = ctx.n, ctx.L + 1, ctx.L
    primes = ctx.primes()
    limb = n * 8
    dnum = -(-ctx.n_q // -(-ctx.n_q // MICRO.dnum))
    ksk = dnum * 2 * (cap + ctx.n_p) * limb
    gen = torch.Generator(device=dev).manual_seed(2)
    out = {}
    for B in (1, 8):
        x = torch.empty((B, 2, cap, n), dtype=torch.int64, device=dev)
        for i in range(cap):
            x[:, :, i] = torch.randint(0, primes[i], (B, 2, n), generator=gen, dtype=torch.int64, device=dev)
        a = secpe.CtBatch(x, L, ctx.scale)
        o = secpe.CtBatch(torch.zeros_like(x), 0, ctx.scale)
        for _ in range(3):
            secpe.keyswitch_batch(ctx, keys, 0, a, o)
        reps = max(10, steps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            secpe.keyswitch_batch(ctx, keys, 0, a, o)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        alg = B * 3 * cap * limb + ksk
        out["B%d" % B] = {"GBps": alg / (ms / 1e3) / 1e9, "ms": ms, "alg_bytes": alg}
        del x, a, o
    out["note"] = ("primitive set N=2^16, 24x50-bit + 4x60-bit special, dnum=3, relinearisation key, top level; "
                   "algorithmic bytes = input + key + output; the key (84 MiB) is L2-sized, so back-to-back "
                   "launches can reuse it from L2")
    keys.close()
    ctx.close()
    return out


def _time_ms(torch, fn, reps):
    """Mean milliseconds of fn() over reps launches (CUDA events on the current stream)."""
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _graph_of(torch, fn):
    """fn captured once as a CUDA graph (after one eager warm-up call); returns its replay."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g.replay


def word_size_probe(secpe, torch, dev, steps):
    """The word-size lever: the negacyclic NTT (forward + inverse) on the
    64-bit residues of argmax8 (q0 60-bit + 23 x 50-bit, 1210 bits) against
    32-bit residues of the word32 chain (29-bit primes, 42 limbs = 1218 bits),
    16 polynomials each (192 / 168 MiB, above L2), and the 32-bit fast base
    conversion of a 14-limb digit (406 bits, like argmax8's 8 x 50-bit digit)
    to 42 primes for 16 items.  Uniform residues (seed 3)."""
    from paper_2502_00847_gb300.presets import ARGMAX8, WORD32
    import dataclasses
    n, polys = 1 << 16, 16
    reps = max(5, steps)
    gen = torch.Generator(device=dev).manual_seed(3)
    out = {}
    ctx = secpe.Context.from_params(ARGMAX8)
    p64 = ctx.primes()[:ctx.n_q]
    bits64 = sum(int(q).bit_length() for q in p64)
    idx64 = list(range(ctx.n_q)) * polys
    x64 = torch.empty((len(idx64), n), dtype=torch.int64, device=dev)
    for r, i in enumerate(idx64):
        x64[r] = torch.randint(0, p64[i], (n,), generator=gen, dtype=torch.int64, device=dev)

    def fi64():
        secpe.ntt(ctx, x64, idx64)
        secpe.ntt(ctx, x64, idx64, inverse=True)
    ms64 = _time_ms(torch, fi64, reps)
    nq64 = ctx.n_q
    del x64
    # 64-bit key switching of 8 ciphertexts' second polynomials at the top level (relinearisation key)
    keys = secpe.Keys(ctx, 3, [])
    xk = torch.empty((8, 2, ctx.n_q, n), dtype=torch.int64, device=dev)
    for i in range(ctx.n_q):
        xk[:, :, i] = torch.randint(0, p64[i], (8, 2, n), generator=gen, dtype=torch.int64, device=dev)
    ak = secpe.CtBatch(xk, ctx.L, ctx.scale)
    ok_ = secpe.CtBatch(torch.zeros_like(xk), 0, ctx.scale)
    msk64 = _time_ms(torch, lambda: secpe.keyswitch_batch(ctx, keys, 0, ak, ok_), reps)
    bitsk64 = bits64 + sum(int(q).bit_length() for q in ctx.primes()[ctx.n_q:])
    del xk, ak, ok_
    keys.close()
    ctx.close()
    q32, sp32 = secpe.select_primes(**dataclasses.asdict(WORD32))
    t = secpe.Ntt32(q32 + sp32)
    l32 = 42
    bits32 = sum(int(q).bit_length() for q in q32[:l32])
    idx32 = list(range(l32)) * polys
    x32 = torch.empty((len(idx32), n), dtype=torch.int32, device=dev)
    for r, i in enumerate(idx32):
        x32[r] = torch.randint(0, q32[i], (n,), generator=gen, dtype=torch.int64, device=dev).to(torch.int32)

    def fi32():
        t.ntt(x32, idx32)
        t.ntt(x32, idx32, inverse=True)
    ms32 = _time_ms(torch, fi32, reps)
    del x32
    for name, ms, limbs, bits, word in (("ntt64", ms64, nq64, bits64, 8), ("ntt32", ms32, l32, bits32, 4)):
        nl = limbs * polys
        out[name] = {"ms_fwd_inv": ms, "limbs": nl, "modulus_bits": bits, "us_per_limb": 1e3 * ms / nl,
                     "ns_per_kbit_coeff": 1e6 * ms / (polys * bits * n / 1000),
                     "GBps": 4 * nl * n * word / (ms / 1e3) / 1e9}
    out["ntt_speedup_per_modulus_bit"] = out["ntt64"]["ns_per_kbit_coeff"] / out["ntt32"]["ns_per_kbit_coeff"]
    B, src, dst = 16, list(range(14)), list(range(14, 48)) + list(range(48, 56))
    xin = torch.empty((B, len(src), n), dtype=torch.int32, device=dev)
    for i in src:
        xin[:, i] = torch.randint(0, q32[i], (B, n), generator=gen, dtype=torch.int64, device=dev).to(torch.int32)
    xo = torch.empty((B, len(dst), n), dtype=torch.int32, device=dev)
    msb = _time_ms(torch, lambda: t.bconv(xin, src, xo, dst), reps)
    alg = B * (len(src) + len(dst)) * n * 4
    out["bconv32"] = {"ms": msb, "items": B, "n_in": len(src), "n_out": len(dst), "GBps": alg / (msb / 1e3) / 1e9,
                      "ns_per_output_limb": 1e6 * msb / (B * len(dst))}
    del xin, xo
    # 32-bit key switching of 8 polynomials: 40 q primes (1,160 bits), 16 special (464 bits), digits of 14 primes
    # (406 bits, dnum 3), against argmax8's 24 q (1,221 bits), 8 special (480 bits), digits of 8 x 50 bits
    qi, pi = list(range(40)), list(range(40, 56))
    allp = q32 + sp32
    bitsk32 = sum(int(allp[i]).bit_length() for i in qi + pi)
    key32 = torch.empty((3, 2, 56, n), dtype=torch.int32, device=dev)
    for i in range(56):
        key32[:, :, i] = torch.randint(0, allp[i], (3, 2, n), generator=gen, dtype=torch.int64,
                                       device=dev).to(torch.int32)
    d32 = torch.empty((8, 40, n), dtype=torch.int32, device=dev)
    for i in qi:
        d32[:, i] = torch.randint(0, allp[i], (8, n), generator=gen, dtype=torch.int64, device=dev).to(torch.int32)
    o32 = torch.empty((8, 2, 40, n), dtype=torch.int32, device=dev)
    # timed as CUDA-graph replays: the call builds its constant tables on the host every time (a probe
    # without a plan object), which would otherwise leave the GPU idle between its launches
    msk32u = _time_ms(torch, _graph_of(torch, lambda: t.keyswitch(d32, qi, pi, 14, key32, o32, False)), reps)
    msk32 = _time_ms(torch, _graph_of(torch, lambda: t.keyswitch(d32, qi, pi, 14, key32, o32, True)), reps)
    del key32, d32, o32
    out["keyswitch"] = {"ms_64bit_B8": msk64, "ms_32bit_B8": msk32, "ms_32bit_unfused_B8": msk32u,
                        "bits_64bit": bitsk64, "bits_32bit": bitsk32,
                        "speedup_per_modulus_bit": (msk64 / bitsk64) / (msk32 / bitsk32),
                        "speedup_per_modulus_bit_unfused": (msk64 / bitsk64) / (msk32u / bitsk32),
                        "note": "64-bit: the fused key switch (secpe_keyswitch_batch) on argmax8, direct calls; "
                                "32-bit: secpe_keyswitch32 as CUDA-graph replays, ModUp conversion in the column "
                                "pass and the inner product in the row pass (unfused: separate INTT, FastBConv, "
                                "NTT and inner-product launches); ModDown unfused in both 32-bit forms"}
    out["note"] = ("NTT: forward + inverse, algorithmic bytes 4 x limbs x N x word (read + write per transform); "
                   "bconv32: input + output bytes; 64-bit reference is the library's secpe_ntt on argmax8 primes")
    t.close()
    return out


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
                                                           "alg_bytes": kp["bytes"],
                                                           "model_bytes": kp["model_bytes"],
                                                           "mul32": kp["mul32"], "ms": kp["total_ms"]}
        if "rotate" in ops:
            per = []
            for j in range(16):
                per.append(timed(lambda: secpe.rotate_batch(ctx, keys, a, 1 << j, o)))
            res["rotate_B%d" % B] = {"ms_mean": sum(per) / len(per), "ms_by_log2_step": per}
        del x, y, out
        torch.cuda.empty_cache()
    if "word32" in ops:
        # the word-size probe (32-bit against 64-bit residues), as in the default run's `word_size`
        res["word_size"] = word_size_probe(secpe, torch, "cuda", args.steps)
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


def serve_rate(ctx, keys, tkeys, views, queries, lam, seconds, seed, budget_bytes, max_batch, max_queries,
               plain=True):
    """One arrival rate of the serving loop.  Poisson arrivals at `lam`/s for
    `seconds` (at most max_queries), each a query drawn from `queries` (its
    input ciphertexts `views` resident on the device, its key set tkeys[i]).

    served: secpe_server_* with continuous batching and admission by the HBM
    budget; latency = arrival -> z ready on the device (host clock).
    plain:  the same arrivals served for real by the plain path, one query
    per call (aggregate + encrypted_argmax) in arrival order on the same GPU;
    latency = arrival -> that call's completion."""
    import torch
    from paper_2502_00847_gb300 import secpe
    rng = np.random.default_rng(seed)
    nq = max(1, min(max_queries, int(round(lam * seconds))))
    arrivals = np.cumsum(rng.exponential(1.0 / lam, nq))
    pick = rng.integers(0, len(queries), nq)
    srv = secpe.Server(ctx, keys, hbm_budget_bytes=budget_bytes, max_batch=max_batch)
    zbufs, pending, lat, batch_sizes, inflight = {}, {}, [], [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nxt = 0
    while nxt < nq or pending:
        now = time.perf_counter() - t0
        while nxt < nq and arrivals[nxt] <= now:
            i = int(pick[nxt])
            z = ctx.new_ct()
            tk = srv.submit(views[i], queries[i].C, queries[i].d_min, queries[i].d_max, queries[i].qseed + nxt, z,
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
            if len(inflight) > 4:   # bounds how far the host runs ahead of the GPU
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
    lat = np.array(lat)
    out = {"rate_qps": lam, "queries": nq, "arrival_window_s": float(arrivals[-1]),
           "served": {"throughput_qps": nq / wall, "p50_ms": 1e3 * float(np.median(lat)),
                      "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                      "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0}}
    if plain:
        zt = ctx.new_ct()
        plat = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, i in zip(arrivals, pick):
            i = int(i)
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            y = secpe.ensemble_aggregate(ctx, views[i], queries[i].d_min, queries[i].d_max)
            secpe.encrypted_argmax(ctx, tkeys[i], y, queries[i].C, queries[i].qseed, out=zt)
            torch.cuda.synchronize()
            plat.append(time.perf_counter() - t0 - a)
        pwall = time.perf_counter() - t0
        plat = np.array(plat)
        out["plain"] = {"throughput_qps": nq / pwall, "p50_ms": 1e3 * float(np.median(plat)),
                        "p99_ms": 1e3 * float(np.percentile(plat, 99)),
                        "note": "run for real: one query per call in arrival order"}
    return out


def run_serve(args, rank):
    """Serving loop (config 5): Poisson arrivals at each rate, continuous
    batching by secpe_server_*, admission by an HBM budget, against the plain
    path run for real on the same arrivals."""
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
    results = []
    for k, lam in enumerate(float(x) for x in args.rates.split(",")):
        results.append(serve_rate(ctx, tenants[0], tkeys, views, pool, lam, args.serve_seconds, 5 + int(lam),
                                  int(args.budget_gb * 1e9), 64, args.serve_queries,
                                  plain=not args.no_plain_serve))
    if rank == 0:
        print(json.dumps({"mode": "serve", "metric": METRIC,
                          "config": {"workload": "serving loop: Poisson arrivals, %.0f s per rate (at most %d "
                                                 "queries), queries from a pool of 64 (K~U{4,8,16}, "
                                                 "C~U{2,3,4,6,14,64}, seed 5), N=2^16, HBM budget %.0f GB, max "
                                                 "batch 64, %d tenant key set(s) resident"
                                                 % (args.serve_seconds, args.serve_queries, args.budget_gb,
                                                    args.tenants),
                                     "tenants": args.tenants},
                          "rates": results}))


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
