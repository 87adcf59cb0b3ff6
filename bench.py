#!/usr/bin/env python3
"""Benchmark of the encrypted logistic-regression worker step on GB300.

Workload (one step): the encrypted gradient step of Eq. 7-8 with the Table 2
binomial polynomial, over 4096 synthetic samples x 784 features (~80% zeros,
values in (0,1], planted-model labels), packed 8 samples per ciphertext at
N = 2^14 with eight ~40-bit limbs, two 59-bit special primes and scale 2^40:
512 data ciphertexts; a step is 1537 relinearised multiplications (three per
data ciphertext and one for the gradient sum) and 14862 rotations in 1538
hoisted rotate-and-sum stages (15, 7 and 7 rotations per data ciphertext, two
stages of 7 after the sum).

Our arm times K steps on the device with CUDA events on the context's stream
(inputs resident in HBM, 1 GB of ciphertexts per step, well above L2); the
e2e figure moves the step's input ciphertexts host->device from pinned memory
and reads the result back, through the C ABI, every step.  The reference arm
(--impl reference) times the CPU oracle on a bounded sample of the same step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "HE mul+relin+rescale/s and enc-LR grad steps/s, batched vs plain, 1 GB300"
# Two 59-bit special primes (digits of two limbs, dnum 4): log2(QP) < 8*40 + 2*59 = 438,
# the 128-bit bound at N = 2^14, and a key switch ~30% cheaper than with one.
LOG_N, L, LIMB_BITS, ALPHA, SPECIAL_BITS, SCALE = 14, 8, 40, 2, 59, 2.0 ** 40
N_SAMPLES, N_FEATURES, G = 4096, 784, 8
# The mask scale sets the scale of the polynomial's result (2^53 here) so that
# the smallest constant, c3 * lr = 4.9e-8, is still encoded with ~2^28 of
# relative precision; the mask itself keeps 2^24 (value (2^27/8) cos(...)).
MASK_SCALE = 2.0 ** 27
WORKLOAD = ("enc-LR gradient step (Eq. 7-8, Table 2 binomial): N=2^14, 8x40-bit limbs + 2x59-bit "
            "special primes (dnum 4), scale 2^40; 4096 samples x 784 features, 8 samples per ciphertext "
            "(512 data ciphertexts); one step = 1537 relinearised multiplications (3 per data ciphertext + 1 "
            "for the gradient sum), 512 tensor accumulations and 14862 rotations in 1538 hoisted "
            "rotate-and-sum stages")


def rot_steps(n_slots: int, g: int) -> list[int]:
    import paper_2006_10091_gb300 as he
    return he.lr_rot_steps(n_slots, g)


def table2_binomial():
    path = os.path.join(ROOT, "tests", "golden", "table2_gradient_polynomials.txt")
    for line in open(path):
        if line.startswith("binomial"):
            return [float(v) for v in line.split()[1:]]
    raise RuntimeError("Table 2 row missing")


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.uuid = device_uuid
        self.proc = None
        # raw samples: $HE_BENCH_CLOCKS_DIR if set, else the system's temporary directory
        out_dir = os.environ.get("HE_BENCH_CLOCKS_DIR") or __import__("tempfile").gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# Integer-pipe roof: the rate of a register-resident chain of 64-bit Shoup
# products (he_probe_alu kind 1), measured on the GPU at the start of the run
# (ALU_PEAK below is replaced by that measurement); the fallback is 152 SMs x
# 2070 MHz x 3.69 products per clock per SM (64 IMAD slots / 17.3 per product,
# an earlier measurement on this kind of GPU): 1.16 T modular products/s.  A
# butterfly is one product; the key-switching kernels also count their
# basis-conversion and inner-product products.
ALU_MODMUL_PEAK = 152 * 2.070e9 * 64 / 17.3
ALU_PEAK = {"per_second": ALU_MODMUL_PEAK, "note": "fallback: 152 SMs x 2070 MHz x 64 IMAD/clk / 17.3 IMAD slots "
                                                  "per 64-bit Shoup product",
            # 64 x 64 -> 128-bit multiply-accumulates (he_probe_alu kind 3); fallback: the Shoup rate
            "mac_per_second": ALU_MODMUL_PEAK, "mac_note": "fallback: the Shoup-product rate",
            # split key products, three 32 x 32 -> 64-bit multiply-adds each (kind 4); fallback: the Shoup rate
            "mac3_per_second": ALU_MODMUL_PEAK, "mac3_note": "fallback: the Shoup-product rate",
            # radix-8 rounds of the lazy butterfly in registers (kind 2): the practical ceiling of a transform
            "butterfly_per_second": None}


def measure_alu_peak(he) -> None:
    """Replace the fallback integer roofs by this GPU's measured rates."""
    try:
        r = he.he_probe_alu(1)
        ALU_PEAK["per_second"] = r["per_second"]
        ALU_PEAK["note"] = (f"measured: register-resident 64-bit Shoup product chain on this GPU "
                            f"({r['per_clock_per_sm']:.2f} per clock per SM)")
        m = he.he_probe_alu(3)
        ALU_PEAK["mac_per_second"] = m["per_second"]
        ALU_PEAK["mac_note"] = (f"measured: register-resident 64x64->128-bit multiply-accumulate chain "
                                f"({m['per_clock_per_sm']:.2f} per clock per SM)")
        m3 = he.he_probe_alu(4)
        ALU_PEAK["mac3_per_second"] = m3["per_second"]
        ALU_PEAK["mac3_note"] = (f"measured: register-resident split key-product chain, three 32x32->64-bit "
                                 f"multiply-adds each ({m3['per_clock_per_sm']:.2f} per clock per SM)")
        ALU_PEAK["butterfly_per_second"] = he.he_probe_alu(2)["per_second"]
    except Exception:  # keep the fallbacks
        return


ALU_CLASSES = ("ntt", "intt", "ks_modup_ntt", "ks_ntt_rot_products", "moddown_ntt", "moddown_ntt_combine",
               "moddown_rescale_ntt", "moddown_rescale_ntt_combine", "rescale_ntt", "rescale_ntt_final")
# DRAM bytes per algorithmic byte of the hoisted stage's row kernel, from an
# ncu capture of one 7-rotation stage over 64 ciphertexts at level 7: 555.7 MB
# of DRAM traffic against 577.8 MB of algorithmic bytes (511.7 MB of
# ciphertext limbs read -- digits and part 0 -- and accumulators written,
# 66.1 MB of the seven keys read once); its traffic grows with the
# ciphertexts, so the roofline scales the launch's algorithmic bytes by it.
KS_ROT_TRAFFIC_PER_ALG_BYTE = 555.7 / 577.8


def roof_time(p: dict, hbm_peak: float, name: str | None = None) -> float:
    """Seconds the class's work takes at its roof: max(weighted integer-pipe
    time, HBM time) for the integer classes (the transform and key-switching
    kernels and the tensor product's products), the HBM time for the rest."""
    work, mac, bfly, by = p["work"], p.get("mac", 0.0), p.get("bfly", 0.0), p["bytes"]
    mac3 = p.get("mac3", 0.0)
    r_bfly = ALU_PEAK["butterfly_per_second"] or ALU_PEAK["per_second"]
    other = max(work - mac - mac3 - bfly, 0.0)
    t_alu = (bfly / r_bfly + other / ALU_PEAK["per_second"] + mac / ALU_PEAK["mac_per_second"]
             + mac3 / ALU_PEAK["mac3_per_second"])
    return max(t_alu, by / (hbm_peak * 1e9))


def class_roof(p: dict, hbm_peak: float, peak_kind: str, name: str, integer: bool | None = None) -> dict:
    """Roofline of one kernel class (or of several summed): the launch time
    against max(integer-pipe time, HBM time).  The integer-pipe time weighs
    each kind of work at its own measured register-resident rate: NTT
    butterflies at the radix-8 lazy butterfly chain (he_probe_alu kind 2),
    Shoup/Barrett products (conversions, scalings, reductions) at the Shoup
    product chain (kind 1), the unreduced 128-bit key products at the
    multiply-accumulate chain (kind 3) and the split key products at their own
    chain (kind 4).  `frac_shoup_only` is the single-rate figure (every unit
    of work at the Shoup rate)."""
    t = p["ms"] * 1e-3
    work, mac, bfly, by = p["work"], p.get("mac", 0.0), p.get("bfly", 0.0), p["bytes"]
    mac3 = p.get("mac3", 0.0)
    r_bfly = ALU_PEAK["butterfly_per_second"] or ALU_PEAK["per_second"]
    other = max(work - mac - mac3 - bfly, 0.0)
    t_alu = (bfly / r_bfly + other / ALU_PEAK["per_second"] + mac / ALU_PEAK["mac_per_second"]
             + mac3 / ALU_PEAK["mac3_per_second"])
    t_hbm = by / (hbm_peak * 1e9)
    gbs = by / t / 1e9 if t > 0 else 0.0
    base = {"kernel": name, "per_launch_ms": p["ms"] / max(1, p["launches"]), "launches": p["launches"],
            "algorithmic_gbs": gbs, "hbm_frac": gbs / hbm_peak, "traffic": None}
    if integer is None:
        integer = name in ALU_CLASSES
    if integer and work > 0:
        if t_alu >= t_hbm:
            rate = work / t if t > 0 else 0.0
            peak = work / t_alu if t_alu > 0 else ALU_PEAK["per_second"]
            base.update({"bound": "alu", "achieved": rate / 1e9, "peak": peak / 1e9, "unit": "G modmul/s",
                         "frac": t_alu / t if t > 0 else 0.0,
                         "frac_shoup_only": rate / ALU_PEAK["per_second"],
                         "work_mix": {"butterflies": bfly, "shoup_products": other, "macs": mac,
                                      "split_macs": mac3},
                         "peak_note": (f"weighted integer roof: {bfly:.3g} butterflies at the measured radix-8 "
                                       f"lazy butterfly chain ({r_bfly / 1e9:.0f} G/s), {other:.3g} Shoup/Barrett "
                                       f"products at {ALU_PEAK['note']} ({ALU_PEAK['per_second'] / 1e9:.0f} G/s), "
                                       f"{mac:.3g} 128-bit key multiply-accumulates at {ALU_PEAK['mac_note']} "
                                       f"({ALU_PEAK['mac_per_second'] / 1e9:.0f} G/s), {mac3:.3g} split key "
                                       f"products at {ALU_PEAK['mac3_note']} "
                                       f"({ALU_PEAK['mac3_per_second'] / 1e9:.0f} G/s)")})
            if name in ("ntt", "intt"):  # butterflies alone against their chain
                base["butterfly_chain_frac"] = (bfly / t) / r_bfly if t > 0 else 0.0
            return base
    base.update({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                 "peak_note": f"{peak_kind} HBM copy bandwidth"})
    return base


def roofline(prof: dict, hbm_peak: float, peak_kind: str):
    """Dominant kernel class by device time -> achieved vs its roof (the
    integer pipe, weighted, for the transform and key-switching kernels; HBM
    for the rest, whichever bounds it)."""
    if not prof:
        return None
    name = max(prof, key=lambda k: prof[k]["ms"])
    r = class_roof(prof[name], hbm_peak, peak_kind, name)
    if name == "ks_ntt_rot_products":
        r["traffic"] = KS_ROT_TRAFFIC_PER_ALG_BYTE * prof[name]["bytes"] / max(1, prof[name]["launches"])
        r["traffic_note"] = ("DRAM bytes per launch: the launch's algorithmic bytes times the DRAM/algorithmic "
                             "ratio of an ncu capture of a smaller launch of the same kernel")
    return r


# ----------------------------------------------------------------------------- ranks

def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over the ranks (each rank runs its own
    independent step: the job takes as long as its slowest rank); a barrier
    follows so that no rank starts its next timed region early."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def weak_scaling_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


# ----------------------------------------------------------------------------- our arm

def build_inputs(he, ctx, data, level):
    n_slots = ctx.n // 2
    zs = __import__("paper_2006_10091_gb300.workloads", fromlist=["x"]).pack_samples(
        data.X, data.y, n_slots, G)
    Z = ctx.new_ct(level, len(zs))
    for k, v in enumerate(zs):
        he.he_encode_encrypt(ctx, v, SCALE, level, Z[k], cid=1000 + k)
    from paper_2006_10091_gb300 import workloads
    W = ctx.new_ct(level)
    he.he_encode_encrypt(ctx, workloads.pack_weights(data.w0, n_slots, G), SCALE, level, W, cid=999)
    return Z, W


def run_ours(args, rank: int, world: int):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_10091_gb300 as he
    measure_alu_peak(he)
    from paper_2006_10091_gb300 import workloads
    from tests.lr_reference import lr_step_fp64

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n_slots = (1 << LOG_N) // 2
    ctx = he.Context(LOG_N, L, LIMB_BITS, ALPHA, SPECIAL_BITS, SCALE, seed=rank,
                     rot_steps=rot_steps(n_slots, G), stream=stream.cuda_stream)
    data = workloads.LRData(seed=rank, n_samples=N_SAMPLES, n_features=N_FEATURES)
    coeffs = table2_binomial()
    lr = 1.0 / N_SAMPLES
    cfg = he.lr_config(coeffs, lr, G, MASK_SCALE)
    tuned = he.he_autotune(ctx, L - 1, 64)  # kernel knobs by timing, before any timed step
    for kv in args.tune or []:  # explicit knobs override the autotuner's
        key, val = kv.split("=")
        he.he_set_tuning(ctx, key, float(val))
        tuned[key] = float(val)
    if args.chunk_bytes:
        he.he_set_tuning(ctx, "chunk_bytes", args.chunk_bytes)
    Z, W = build_inputs(he, ctx, data, L)
    out = ctx.new_ct(L)
    if args.graph:  # the same step through the workers entry point, replayed as one CUDA graph
        step = lambda: he.he_lr_gradient_step_workers(ctx, [(Z, W, out)], cfg, graph=True)  # noqa: E731
    else:
        step = lambda: he.he_lr_gradient_step(ctx, Z, W, cfg, out)  # noqa: E731

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # accuracy of the step this bench times (decrypt vs FP64 Eq. 7-8)
    got = he.he_decrypt_decode(ctx, out)
    want = workloads.pack_weights(lr_step_fp64(data.X, data.y, data.w0, coeffs, lr), n_slots, G)
    rel_err = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            torch.cuda.nvtx.range_push("lr_step")  # lets ncu capture exactly the timed steps
            step()
            torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_per_step = ms / args.steps

    # kernel-class timing over a profiled region of the same step
    he.he_profile_enable(ctx, True)
    prof_steps = max(1, min(3, args.steps))
    for _ in range(prof_steps):
        step()
    prof = {k: he.he_profile_read(ctx, k) for k in he.he_profile_names(ctx)}
    he.he_profile_enable(ctx, False)
    hbm_peak, peak_kind = measured_peaks()
    roof = roofline(prof, hbm_peak, peak_kind)
    kernels = {k: {"launches_per_step": v["launches"] // prof_steps, "ms_per_step": v["ms"] / prof_steps}
               for k, v in prof.items()}

    # e2e: host->device copy of the step's inputs (pinned), the step, result read back
    nZ = len(Z)
    host_in = torch.empty((nZ, 2, L, ctx.n), dtype=torch.int64, pin_memory=True)
    host_w = torch.empty((1, 2, L, ctx.n), dtype=torch.int64, pin_memory=True)
    host_out = torch.empty((2, L - 5, ctx.n), dtype=torch.int64, pin_memory=True)
    he.he_ct_export_batch(ctx, Z, host_in)
    he.he_ct_export_batch(ctx, [W], host_w)
    # the public host-buffer entry point: copies of the data ciphertexts run on
    # a second stream, overlapped with the circuit chunk by chunk
    host_step = lambda: he.he_lr_gradient_step_host(ctx, host_in, L, SCALE, host_w[0], L, SCALE, cfg,  # noqa: E731
                                                    host_out)
    host_step()  # grows the device input buffer
    e2e_steps = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    got_e2e = host_out.numpy().view(np.uint64)
    # this box's pinned host-to-device bandwidth (one copy of the step's
    # inputs, alone): the e2e figure depends on it, and it varies by box
    dev_in = torch.empty(host_in.shape, dtype=host_in.dtype, device=dev)
    dev_in.copy_(host_in, non_blocking=True)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    dev_in.copy_(host_in, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = host_in.numel() * 8 / (c0.elapsed_time(c1) * 1e-3) / 1e9
    del dev_in
    he.he_lr_gradient_step(ctx, Z, W, cfg, out)
    e2e_same = bool(np.array_equal(got_e2e, he.he_ct_export(ctx, out)))
    h2d = (nZ + 1) * 2 * L * ctx.n * 8
    d2h = 2 * (L - 5) * ctx.n * 8

    extra = {}
    if not args.quick and rank == 0:
        extra.update(hmult_rates(he, torch, stream))
        extra["batched_workers"] = batched_workers(he, torch, stream)
        extra["serving"] = serving(he, torch, stream)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(data, coeffs, lr)
    value = weak_scaling_value(1.0, world, ms_per_step * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": 1 << LOG_N, "limbs": L, "special_primes": ALPHA,
                   "scale_log2": 40, "samples": N_SAMPLES, "features": N_FEATURES,
                   "samples_per_ciphertext": G, "data_ciphertexts": nZ,
                   "l2": "inputs larger than L2 (1.07 GB of ciphertexts per step)",
                   "scratch_budget_bytes": int(args.chunk_bytes) if args.chunk_bytes else None,
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "accuracy": {"max_rel_err_vs_fp64": rel_err, "gate": 2.0 ** -20, "ok": rel_err < 2.0 ** -20},
        "e2e": {"value": weak_scaling_value(1.0, world, e2e_s), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "he_lr_gradient_step_host (pinned host buffers)",
                "h2d_gbs_measured": h2d_gbs,
                "same_residues_as_device_step": e2e_same},
        "gpu_launches": int(sum(v["launches"] for v in prof.values()) // prof_steps),
        "autotune": tuned,
        "roofline": roof, "kernels": kernels, "clocks": clk.summary(), "cpu_baseline": cpu,
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))


def hmult_rates(he, torch, stream):
    """mul+relin+rescale/s at the small (N=2^12, 3 limbs, 16 pairs) and large
    (N=2^16, 24 limbs + 4 special primes, dnum 6, 64 ciphertexts)
    configurations, batched (one call) and plain (one call per pair)."""
    from paper_2006_10091_gb300 import workloads
    out = {}
    for name, (log_n, nl, bits, alpha, sbits, scale, count) in {
            "hmult_small": (12, 3, 40, 1, 60, 2.0 ** 30, 16),
            "hmult_large": (16, 24, 50, 4, 60, 2.0 ** 50, 64)}.items():
        rots = []
        if name == "hmult_large":
            rots = [1 << t for t in range(10)]
            rots += [r for st in he.rotsum_stages(1, 10) for r in st if r not in rots]
        ctx = he.Context(log_n, nl, bits, alpha, sbits, scale, seed=0, stream=stream.cuda_stream, rot_steps=rots)
        tuned = he.he_autotune(ctx, nl, 16) if name == "hmult_large" else None
        n = 1 << log_n
        A, B, O = ctx.new_ct(nl, count), ctx.new_ct(nl, count), ctx.new_ct(nl, count)
        for i in range(count):
            he.he_encode_encrypt(ctx, workloads.uniform_slots(2 * i, n // 2), scale, nl, A[i], cid=2 * i)
            he.he_encode_encrypt(ctx, workloads.uniform_slots(2 * i + 1, n // 2), float(ctx.primes[nl - 1]),
                                 nl, B[i], cid=2 * i + 1)
        for _ in range(3):
            he.he_mul_relin_rescale_batch(ctx, A, B, O)
        torch.cuda.synchronize()
        reps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            he.he_mul_relin_rescale_batch(ctx, A, B, O)
        e1.record(stream)
        torch.cuda.synchronize()
        batched = count * reps * 1000.0 / e0.elapsed_time(e1)
        e0.record(stream)
        for _ in range(reps):
            for i in range(count):
                he.he_mul_relin_rescale(ctx, A[i], B[i], O[i])
        e1.record(stream)
        torch.cuda.synchronize()
        plain = count * reps * 1000.0 / e0.elapsed_time(e1)
        got = he.he_decrypt_decode(ctx, O[0])
        want = workloads.uniform_slots(0, n // 2) * workloads.uniform_slots(1, n // 2)
        err = float(np.max(np.abs(got - want)))
        out[name] = {"per_s_batched": batched, "per_s_plain": plain, "count": count, "N": n, "limbs": nl,
                     "max_abs_err": err,
                     "second_operand_scale": "q_{l-1} (the product returns to the first operand's scale)"}
        if name == "hmult_small":
            # the configuration as stated: both operands at scale 2^30, so the
            # product is left at 2^60 / q_{l-1} ~ 2^20 after the rescale
            b2 = ctx.new_ct(nl)
            he.he_encode_encrypt(ctx, workloads.uniform_slots(1, n // 2), scale, nl, b2, cid=1)
            o2 = ctx.new_ct(nl)
            he.he_mul_relin_rescale(ctx, A[0], b2, o2)
            got2 = he.he_decrypt_decode(ctx, o2)
            out[name]["both_operands_at_2^30"] = {
                "max_abs_err": float(np.max(np.abs(got2 - want))), "result_scale_log2": math.log2(o2.scale),
                "gate": 1e-4}
        if name == "hmult_large":
            # 1024-slot rotate-and-sum over the 64: hoisted stages (five of rotations
            # by s, 2s, 3s), and as ten rotations by 1, 2, ..., 512 with additions
            T = ctx.new_ct(nl, count)
            stages = he.rotsum_stages(1, 10)

            def rotsum():
                for st in stages:
                    he.he_rotate_sum_batch(ctx, O, st, T)
                    O[:], T[:] = T[:], O[:]

            def rotsum_sequential():
                for t in range(10):
                    he.he_rotate_batch(ctx, O, 1 << t, T)
                    for i in range(count):
                        he.he_add(ctx, O[i], T[i], O[i])
            for fn, key in ((rotsum, "rotate_and_sum_per_s"), (rotsum_sequential, "rotate_and_sum_sequential_per_s")):
                fn()
                torch.cuda.synchronize()
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                out[name][key] = count * 1000.0 / e0.elapsed_time(e1)
            out[name]["rotate_and_sum_stages"] = [list(st) for st in stages]
            out[name]["autotune"] = tuned
            out[name]["roofline"] = large_rooflines(he, torch, stream, ctx, A, B, O, T)
        ctx.close()
        del A, B, O
        torch.cuda.empty_cache()
    return out


def large_rooflines(he, torch, stream, ctx, A, B, O, T):
    """Roofline objects at N = 2^16 (24 limbs, four special primes, the
    batch of 64 ciphertexts): the key switch of a rotation by one slot (all its
    kernel classes together and its row kernel alone), of a multiplication,
    and the forward and inverse NTT over the batch's 3072 limbs (1.6 GB, more
    than L2), each from kernel-class timing of one profiled batch."""
    hbm_peak, peak_kind = measured_peaks()
    ks_classes = ("ks_modup_ntt", "ks_ntt_rot_products", "intt", "moddown_ntt", "moddown_ntt_combine",
                  "moddown_rescale_ntt", "moddown_rescale_ntt_combine", "tensor")
    out = {}

    def profiled(fn):
        fn()
        torch.cuda.synchronize()
        he.he_profile_enable(ctx, True)
        fn()
        prof = {k: he.he_profile_read(ctx, k) for k in he.he_profile_names(ctx)}
        he.he_profile_enable(ctx, False)
        return prof

    def summed(prof, names):
        keys = [k for k in names if k in prof]
        return {f: sum(prof[k][f] for k in keys) for f in ("ms", "work", "mac", "mac3", "bfly", "bytes", "launches")}

    for key, fn in (("keyswitch_rotation", lambda: he.he_rotate_batch(ctx, A, 1, O)),
                    ("mul_relin_rescale", lambda: he.he_mul_relin_rescale_batch(ctx, A, B, O))):
        prof = profiled(fn)
        keys = [k for k in ks_classes if k in prof]
        out[key] = class_roof(summed(prof, ks_classes), hbm_peak, peak_kind, key, integer=True)
        out[key]["classes"] = keys
        # the operation's roof as the sum over its kernels of each one's own
        # roof time (integer pipe, weighted, or HBM, whichever is longer: the
        # tensor product is bound by HBM); `frac` above counts all their work
        # as integer work, which undercounts an HBM-bound kernel's roof
        t_roof = sum(roof_time(prof[k], hbm_peak) for k in keys)
        t_all = sum(prof[k]["ms"] for k in keys) * 1e-3
        out[key]["frac_all_integer"] = out[key]["frac"]
        out[key]["frac"] = t_roof / t_all if t_all > 0 else 0.0
        out[key]["frac_note"] = ("sum over the kernel classes of max(weighted integer-pipe time, HBM time) "
                                 "over their measured time; frac_all_integer: all work as integer work")
        if key == "keyswitch_rotation":
            out["ks_ntt_rot_products"] = class_roof(prof["ks_ntt_rot_products"], hbm_peak, peak_kind,
                                                    "ks_ntt_rot_products")
            out["moddown_ntt_combine"] = class_roof(prof["moddown_ntt_combine"], hbm_peak, peak_kind,
                                                    "moddown_ntt_combine")
    buf = torch.cat([a.tensor.reshape(-1) for a in A]).reshape(len(A) * 2, -1)  # 128 polynomials of 24 limbs
    nl = A[0].level
    for inverse in (False, True):
        fn = lambda: he.he_ntt(ctx, buf, buf.shape[0], nl * ctx.n, nl, 0, inverse)  # noqa: E731
        prof = profiled(fn)
        k = "intt" if inverse else "ntt"
        out[k] = class_roof(prof[k], hbm_peak, peak_kind, k)
    return out


def batched_workers(he, torch, stream, reps=2):
    """32 workers of log-uniform 512..8192 samples x 784 features, weights at
    levels uniform in 2..8 (those below 6 are refreshed to 8 by the in-process
    key holder first): all workers in one graph-replayed batched call vs one
    call per worker (the per-instance path, no cross-worker batching)."""
    from paper_2006_10091_gb300 import workloads
    from tests.lr_reference import lr_step_fp64
    n_slots = (1 << LOG_N) // 2
    ctx = he.Context(LOG_N, L, LIMB_BITS, ALPHA, SPECIAL_BITS, SCALE, seed=0, rot_steps=rot_steps(n_slots, G),
                     stream=stream.cuda_stream)
    sizes = workloads.shard_sizes(0, 32)
    levels = workloads.shard_levels(0, 32)
    coeffs = table2_binomial()
    lr = 1.0 / N_SAMPLES  # one learning rate for all workers
    cfg = he.lr_config(coeffs, lr, G, MASK_SCALE)
    tuned = he.he_autotune(ctx, L, 64)
    shards, datas = [], []
    t0 = time.perf_counter()
    for k, (ns, lv) in enumerate(zip(sizes, levels)):
        data = workloads.LRData(seed=100 + k, n_samples=ns, n_features=N_FEATURES)
        datas.append(data)
        zs = workloads.pack_samples(data.X, data.y, n_slots, G)
        Z = ctx.new_ct(L, len(zs))
        for i, v in enumerate(zs):
            he.he_encode_encrypt(ctx, v, SCALE, L, Z[i], cid=(k << 16) + i)
        W = ctx.new_ct(L)
        he.he_encode_encrypt(ctx, workloads.pack_weights(data.w0, n_slots, G), SCALE, lv, W, cid=(k << 16) + 0xFFFF)
        shards.append((Z, W, ctx.new_ct(L)))
    setup_s = time.perf_counter() - t0
    n_ct = sum(len(z) for z, _, _ in shards)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    he.he_lr_gradient_step_workers(ctx, shards, cfg, refresh_level=L, graph=True)  # capture
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        he.he_lr_gradient_step_workers(ctx, shards, cfg, refresh_level=L, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / reps
    k_check = max(range(32), key=lambda k: sizes[k])
    got = he.he_decrypt_decode(ctx, shards[k_check][2])
    d = datas[k_check]
    want = workloads.pack_weights(lr_step_fp64(d.X, d.y, d.w0, coeffs, lr), n_slots, G)
    rel = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    for sh in shards:  # warm the per-worker path
        he.he_lr_gradient_step_workers(ctx, [sh], cfg, refresh_level=L)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for sh in shards:
            he.he_lr_gradient_step_workers(ctx, [sh], cfg, refresh_level=L)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / reps
    # The plain per-ciphertext path: every worker's circuit evaluated one data
    # ciphertext at a time (each operation a launch over one ciphertext), as a
    # single-instance HE library runs it.  Its cost is linear in the number of
    # data ciphertexts plus a per-worker final stage, so it is timed on the
    # first 4 and first 8 ciphertexts of every worker and extrapolated to the
    # whole shard from those two points.
    he.he_set_tuning(ctx, "lr_chunk", 1)
    pc = {}
    for m in (4, 8):
        sub = [(Z[:m], W, Wo) for Z, W, Wo in shards]
        for sh in sub[:2]:
            he.he_lr_gradient_step_workers(ctx, [sh], cfg, refresh_level=L)
        torch.cuda.synchronize()
        per = []
        for sh in sub:
            e0.record(stream)
            he.he_lr_gradient_step_workers(ctx, [sh], cfg, refresh_level=L)
            e1.record(stream)
            torch.cuda.synchronize()
            per.append(e0.elapsed_time(e1))
        pc[m] = per
    he.he_set_tuning(ctx, "lr_chunk", 0)
    per_ct_ms = []
    plain_ct_ms = 0.0
    for k, (Z, _, _) in enumerate(shards):
        slope = max((pc[8][k] - pc[4][k]) / 4.0, 0.0)
        fixed = max(pc[4][k] - 4 * slope, 0.0)
        per_ct_ms.append(slope)
        plain_ct_ms += fixed + slope * len(Z)
    out = {"workers": 32, "data_ciphertexts": n_ct, "samples": int(sum(sizes)),
           "levels": levels, "refreshed": int(sum(1 for v in levels if v < 6)),
           "batched_ms_per_round": batched_ms,
           "batched_worker_steps_per_s": 32 * 1000.0 / batched_ms,
           # the configuration's own comparison: 32 separate plain calls, one per worker
           "speedup_vs_plain": plain_ms / batched_ms, "target": 3.0, "target_met": plain_ms / batched_ms >= 3.0,
           "per_worker_calls": {"ms_per_round": plain_ms, "worker_steps_per_s": 32 * 1000.0 / plain_ms,
                                "speedup_of_batched": plain_ms / batched_ms,
                                "what": "the plain path: 32 separate calls, one per worker; each call batches "
                                        "its own ciphertexts"},
           "plain_per_ciphertext": {"ms_per_round": plain_ct_ms, "worker_steps_per_s": 32 * 1000.0 / plain_ct_ms,
                                    "role": "second comparison, not the configuration's plain path",
                                    "speedup_of_batched": plain_ct_ms / batched_ms,
                                    "median_ms_per_ciphertext": float(np.median(per_ct_ms)),
                                    "what": "each worker one ciphertext at a time; timed on 4 and 8 ciphertexts "
                                            "per worker, extrapolated linearly to the full shard"},
           "max_rel_err_vs_fp64_largest_worker": rel, "setup_s": setup_s, "autotune": tuned}
    ctx.close()
    del shards
    torch.cuda.empty_cache()
    return out


SERVE_LOG_NS = (13, 14, 15, 16)
SERVE_L, SERVE_BITS, SERVE_ALPHA, SERVE_BATCH = 20, 50, 4, 128
SERVE_SCALE = 2.0 ** 50
# The step's mask scale: the mask's rounding error per slot grows like
# sqrt(N g) / mask_scale, which 2^34 keeps near 1e-7 of the gradient at
# N = 2^16 and 512 samples per ciphertext.
SERVE_MASK_SCALE = 2.0 ** 34
# Steps refresh weights below 7 limbs so that their result keeps two limbs
# (one ~50-bit limb holds only |w| < 1/2 at scale 2^50).
SERVE_MIN_STEP_LEVEL = 7


def serving(he, torch, stream, n_requests=400, n_warm=100, rate=2000.0, seed=0, budget=48 << 30,
            inflight=4, wave=16):
    """A Poisson stream (mean `rate` req/s) of encrypted gradient-step and
    inference requests over ring sizes N = 2^13..2^16 (20 limbs of ~50 bits,
    4 special primes, scale 2^50; at 2^40 the encryption noise summed over
    4096 features at N = 2^16 alone exceeds 2^-20 of the result), weights at
    levels uniform in 2..20 (below what the circuit needs they are refreshed
    in-process first), feature counts log-uniform in 64..4096 padded to a
    power of two, 128 samples per request, kinds 50/50.  The
    continuous-batching server is compared with the same server restricted
    to one request at a time; latency is arrival to completion as the server
    records it."""
    from paper_2006_10091_gb300 import workloads
    from tests.lr_reference import lr_step_fp64
    rng = np.random.default_rng(seed)
    coeffs = table2_binomial()
    t_setup = time.perf_counter()
    ctxs = []
    for log_n in SERVE_LOG_NS:
        n_slots = 1 << (log_n - 1)
        rots = []  # every sample count per ciphertext the feature counts 64..4096 give
        for F in (64 << t for t in range(7)):
            if F <= n_slots:
                rots += [r for r in he.lr_rot_steps(n_slots, n_slots // F) if r not in rots]
        ctxs.append(he.Context(log_n, SERVE_L, SERVE_BITS, SERVE_ALPHA, 60, SERVE_SCALE, seed=0, rot_steps=rots,
                               stream=stream.cuda_stream))
    classes, wbuf, obuf = {}, {}, {}

    def data_class(ci, F):
        key = (ci, F)
        if key not in classes:
            ctx = ctxs[ci]
            n_slots = ctx.n // 2
            g = n_slots // F
            data = workloads.LRData(seed=1000 * ci + F, n_samples=SERVE_BATCH, n_features=F - F // 8)
            zs = workloads.pack_samples(data.X, data.y, n_slots, g)
            Z = ctx.new_ct(SERVE_L, len(zs))
            for i, v in enumerate(zs):
                he.he_encode_encrypt(ctx, v, SERVE_SCALE, SERVE_L, Z[i], cid=(ci << 24) + (F << 8) + i)
            host = torch.empty((len(zs), 2, SERVE_L, ctx.n), dtype=torch.int64, pin_memory=True)
            he.he_ct_export_batch(ctx, Z, host)
            classes[key] = (data, g, host)
        return classes[key]

    def weights(ci, F, wl):
        key = (ci, F, wl)
        if key not in wbuf:
            ctx = ctxs[ci]
            data, g, _ = data_class(ci, F)
            W = ctx.new_ct(wl)
            he.he_encode_encrypt(ctx, workloads.pack_weights(data.w0, ctx.n // 2, g), SERVE_SCALE, wl, W,
                                 cid=(1 << 31) + (ci << 24) + (F << 8) + wl)
            host = torch.empty((1, 2, wl, ctx.n), dtype=torch.int64, pin_memory=True)
            he.he_ct_export_batch(ctx, [W], host)
            wbuf[key] = host
        return wbuf[key]

    reqs = []
    for r in range(n_warm + n_requests):
        ci = int(rng.integers(0, len(SERVE_LOG_NS)))
        f = math.exp(rng.uniform(math.log(64), math.log(4096)))
        F = min(4096, 1 << math.ceil(math.log2(f)))
        kind = he.HE_REQ_GRADIENT if rng.random() < 0.5 else he.HE_REQ_INFERENCE
        wl = int(rng.integers(2, SERVE_L + 1))
        data, g, zh = data_class(ci, F)
        nz = zh.shape[0]
        need = SERVE_MIN_STEP_LEVEL if kind == he.HE_REQ_GRADIENT else 5
        l_out = (wl if wl >= need else SERVE_L) - (5 if kind == he.HE_REQ_GRADIENT else 3)
        # one output buffer per (ring, features, kind), sized for the highest
        # output level; requests of a class overwrite each other's results
        # (accuracy is checked afterwards on requests served alone)
        okey = (ci, F, kind)
        if okey not in obuf:
            top = SERVE_L - (5 if kind == he.HE_REQ_GRADIENT else 3)
            obuf[okey] = torch.empty((nz if kind == he.HE_REQ_INFERENCE else 1) * 2 * top * ctxs[ci].n,
                                     dtype=torch.int64, pin_memory=True)
        cfg = (he.lr_config(coeffs, 1.0 / SERVE_BATCH, g, SERVE_MASK_SCALE) if kind == he.HE_REQ_GRADIENT
               else he.lr_config(coeffs, 1.0, g, SERVE_SCALE))
        reqs.append(dict(ci=ci, F=F, kind=kind, wl=wl, Z=zh, W=weights(ci, F, wl), cfg=cfg, out=obuf[okey],
                         cid=(ci << 24) + (F << 8) + wl, nz=nz, l_out=l_out, need=need))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    arrivals = workloads.poisson_arrivals(seed, rate, n_requests)

    def submit(srv, r):
        return srv.submit(r["ci"], r["kind"], r["Z"], SERVE_L, SERVE_SCALE, r["W"], r["wl"], SERVE_SCALE, r["cfg"],
                          r["out"], refresh_cid=r["cid"], min_w_level=r["need"])

    def run(srv, arr, timed, warm=True):
        if warm:
            for r in reqs[:n_warm]:  # warm-up: plans, masks and workspaces
                submit(srv, r)
            srv.drain(1200)
            srv.poll(cap=n_warm + 16)
        t0 = time.perf_counter()
        for r, ta in zip(timed, arr):
            while True:
                dt = ta - (time.perf_counter() - t0)
                if dt <= 0:
                    break
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
            submit(srv, r)
        t_sub = time.perf_counter() - t0
        srv.drain(1200)
        span = time.perf_counter() - t0
        res = srv.poll(cap=len(timed) + 16)
        stats = srv.stats()
        bad = [x for x in res if x["status"] != 0]
        if bad or len(res) != len(timed):
            codes = sorted({x["status"] for x in bad})
            raise RuntimeError(f"serving: {len(bad)} failed requests (codes {codes}: {srv.last_error()}), "
                               f"{len(res)} of {len(timed)} returned")
        lat = np.array([x["latency_ms"] for x in res])
        return {"requests": len(timed), "offered_per_s": len(timed) / float(arr[len(timed) - 1]),
                "requests_per_s": len(timed) / span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "arrival_window_s": t_sub, "span_s": span, "waves": stats["waves"],
                "peak_running_waves": stats["peak_running"], "peak_device_bytes": stats["peak_used"]}

    timed = reqs[n_warm:]
    srv_c = he.Server(ctxs, budget, max_inflight=inflight, max_wave=wave)
    srv_o = he.Server(ctxs, budget, max_inflight=1, max_wave=1, max_running=1)
    try:
        cont = run(srv_c, arrivals, timed)
        one = run(srv_o, arrivals, timed)
        # the same servers under a load both sustain (80% of the one-at-a-time
        # throughput): latency without a backlog
        n_s = min(150, len(timed))
        arr_s = workloads.poisson_arrivals(seed + 1, 0.8 * one["requests_per_s"], n_s)
        cont_s = run(srv_c, arr_s, timed[:n_s], warm=False)
        one_s = run(srv_o, arr_s, timed[:n_s], warm=False)
    finally:
        srv_c.close()
        srv_o.close()
    # accuracy: the first request of every (ring, kind) class, served alone and decrypted
    acc = {}
    srv = he.Server(ctxs, budget, max_inflight=1, max_wave=1, max_running=1)
    try:
        for ci, ctx in enumerate(ctxs):
            for kind in (he.HE_REQ_GRADIENT, he.HE_REQ_INFERENCE):
                r = next((x for x in reqs if x["ci"] == ci and x["kind"] == kind), None)
                if r is None:
                    continue
                submit(srv, r)
                srv.drain(600)
                info = srv.poll()[0]
                data, g, _ = classes[(ci, r["F"])]
                n_slots = ctx.n // 2
                cnt = 1 if kind == he.HE_REQ_GRADIENT else r["nz"]
                words = 2 * r["l_out"] * ctx.n
                outs = [r["out"][k * words:(k + 1) * words] for k in range(cnt)]
                err = 0.0
                for k, o in enumerate(outs):
                    ct = ctx.new_ct(r["l_out"])
                    he.he_ct_import(ctx, o.numpy().view(np.uint64).reshape(2, r["l_out"], ctx.n), r["l_out"],
                                    info["scale"], ct)
                    got = he.he_decrypt_decode(ctx, ct)
                    if kind == he.HE_REQ_GRADIENT:
                        want = workloads.pack_weights(
                            lr_step_fp64(data.X, data.y, data.w0, coeffs, 1.0 / SERVE_BATCH), n_slots, g)
                        err = max(err, float(np.max(np.abs(got - want)) / np.max(np.abs(want))))
                    else:
                        m = data.y * (data.X @ data.w0)
                        p = coeffs[0] + coeffs[1] * m + coeffs[2] * m * m + coeffs[3] * m ** 3
                        for smp in range(g):
                            if k * g + smp < len(p):
                                err = max(err, float(np.max(np.abs(got[smp::g] - p[k * g + smp]))))
                name = f"N=2^{SERVE_LOG_NS[ci]} {'gradient' if kind == he.HE_REQ_GRADIENT else 'inference'}"
                acc[name] = {"F": r["F"], "w_level": r["wl"], "err": err,
                             "err_kind": "max rel vs FP64" if kind == he.HE_REQ_GRADIENT else "max abs vs FP64"}
    finally:
        srv.close()
    for c in ctxs:
        c.close()
    torch.cuda.empty_cache()
    mix = {"requests": n_requests, "warmup_requests": n_warm, "offered_per_s": rate,
           "rings": {f"2^{SERVE_LOG_NS[i]}": sum(1 for r in reqs[n_warm:] if r["ci"] == i)
                     for i in range(len(SERVE_LOG_NS))},
           "gradient_share": sum(1 for r in reqs[n_warm:] if r["kind"] == he.HE_REQ_GRADIENT) / n_requests,
           "refreshed": sum(1 for r in reqs[n_warm:] if r["wl"] < r["need"]),
           "data_ciphertexts": int(sum(r["nz"] for r in reqs[n_warm:])), "budget_bytes": budget}
    return {"server": {"max_inflight": inflight, "max_wave": wave}, "continuous": cont, "one_at_a_time": one,
            "throughput_ratio": cont["requests_per_s"] / one["requests_per_s"],
            "sustained_load": {"continuous": cont_s, "one_at_a_time": one_s}, "mix": mix, "accuracy": acc,
            "setup_s": setup_s,
            "params": "N=2^13..2^16, 20x50-bit limbs + 4x60-bit special primes (dnum 5), scale 2^50; "
                      "not 128-bit secure at N<=2^15 (benchmark parameters)"}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_step_inputs(o, data, n_ct):
    from paper_2006_10091_gb300 import workloads
    n_slots = (1 << LOG_N) // 2
    zs = workloads.pack_samples(data.X[:n_ct * G], data.y[:n_ct * G], n_slots, G)
    Z = [o.encrypt(o.encode(v), L, cid=1000 + k) for k, v in enumerate(zs)]
    W = o.encrypt(o.encode(workloads.pack_weights(data.w0, n_slots, G)), L, cid=999)
    return Z, W


def _oracle_rate(o, Z, W, coeffs, lr, m):
    """Seconds of the oracle's step over m and over 2m data ciphertexts ->
    (per-ciphertext seconds at this thread count, fixed seconds of the final
    stage); the step over the 512 ciphertexts is extrapolated linearly."""
    t = []
    for k in (m, 2 * m):
        t0 = time.perf_counter()
        o.lr_gradient_step(Z[:k], W, coeffs, lr, G, MASK_SCALE)
        t.append(time.perf_counter() - t0)
    per = max((t[1] - t[0]) / m, 1e-9)
    return per, max(t[0] - m * per, 0.0), t


def cpu_baseline(data, coeffs, lr):
    """The oracle as it stands on a bounded sample of the step, on all host
    cores (OpenMP over the data ciphertexts and over limbs) and on one core:
    the step over m and 2m of the 512 data ciphertexts (m = 1 on one core,
    m = the thread count on all), extrapolated linearly to the 512."""
    import oracle
    nproc = os.cpu_count() or 1
    threads0 = oracle.get_threads()
    o = oracle.Oracle(LOG_N, L, LIMB_BITS, ALPHA, SPECIAL_BITS, SCALE, seed=0,
                      rot_steps=rot_steps((1 << LOG_N) // 2, G))
    n_ct = N_SAMPLES // G
    out = {}
    try:
        for label, nt in (("all", max(1, threads0)), ("one", 1)):
            oracle.set_threads(nt)
            m = 1 if nt == 1 else min(nt, n_ct // 2)
            Z, W = _oracle_step_inputs(o, data, 2 * m)
            per, fixed, t = _oracle_rate(o, Z, W, coeffs, lr, m)
            step_s = fixed + n_ct * per
            out[label] = {"value": 1.0 / step_s, "cores": nt, "sample_s": t, "m": m}
    finally:
        oracle.set_threads(threads0)
    a, one = out["all"], out["one"]
    return {"value": a["value"], "unit": "steps/s", "cores": a["cores"], "kind": "oracle",
            "nproc": nproc, "cpu_model": cpu_model(),
            "sample": (f"the oracle's step over {a['m']} and {2 * a['m']} of the {n_ct} data ciphertexts on "
                       f"{a['cores']} threads ({a['sample_s'][0]:.1f} s, {a['sample_s'][1]:.1f} s), extrapolated "
                       f"linearly; exact __int128 residue arithmetic, OpenMP over ciphertexts and limbs"),
            "one_core": {"value": one["value"], "unit": "steps/s", "cores": 1,
                         "sample": f"the step over 1 and 2 data ciphertexts ({one['sample_s'][0]:.1f} s, "
                                   f"{one['sample_s'][1]:.1f} s), extrapolated linearly"}}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank: int):
    """The oracle as it stands, on the host's cores, on the step this bench
    times: each timed step runs the oracle's step over m data ciphertexts (m =
    the thread count) and extrapolates to the 512 with the fixed final-stage
    cost measured during warm-up (a run over 2m)."""
    if rank != 0:
        return
    import oracle
    from paper_2006_10091_gb300 import workloads
    data = workloads.LRData(seed=0, n_samples=N_SAMPLES, n_features=N_FEATURES)
    coeffs = table2_binomial()
    lr = 1.0 / N_SAMPLES
    o = oracle.Oracle(LOG_N, L, LIMB_BITS, ALPHA, SPECIAL_BITS, SCALE, seed=0,
                      rot_steps=rot_steps((1 << LOG_N) // 2, G))
    threads = oracle.get_threads()
    n_ct = N_SAMPLES // G
    m = min(max(1, threads), n_ct // 2)
    Z, W = _oracle_step_inputs(o, data, 2 * m)
    per, fixed, _ = _oracle_rate(o, Z, W, coeffs, lr, m)  # warm-up: the fixed final-stage cost
    for _ in range(max(0, args.warmup - 2)):
        o.lr_gradient_step(Z[:m], W, coeffs, lr, G, MASK_SCALE)
    step_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.lr_gradient_step(Z[:m], W, coeffs, lr, G, MASK_SCALE)
        t = time.perf_counter() - t0
        step_s.append(fixed + (n_ct / m) * max(t - fixed, 1e-9))
    mean = sum(step_s) / len(step_s)
    value = 1.0 / mean
    sample = (f"each step times the oracle's step over {m} of the {n_ct} data ciphertexts on {threads} threads "
              f"and extrapolates linearly (fixed final-stage cost {fixed:.2f} s from a {2 * m}-ciphertext run)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_micro(args):
    """One kernel class alone: forward/inverse NTT over `--polys` polynomials
    of 8 limbs at N = 2^log_n (more than L2), timed with CUDA events.  Each
    rate is also given as a fraction of the register-resident radix-8 lazy
    butterfly chain (he_probe_alu kind 2: the same butterflies with no memory
    traffic), beside the fraction of the Shoup-product roof."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_10091_gb300 as he
    measure_alu_peak(he)
    bfly_roof = he.he_probe_alu(2)["per_second"]
    from paper_2006_10091_gb300 import workloads
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    log_n, nl = args.log_n, 8
    ctx = he.Context(log_n, nl, LIMB_BITS, 1, SPECIAL_BITS, SCALE, seed=0, stream=stream.cuda_stream)
    n = 1 << log_n
    host = workloads.residues(1, ctx.primes[:nl], n, parts=args.polys)
    t = torch.from_numpy(host.view(np.int64)).cuda()
    out = {}
    for kv in args.tune or []:
        key, val = kv.split("=")
        he.he_set_tuning(ctx, key, float(val))
    for shape, generic, inverse in ((0, False, False), (0, False, True), (1, False, False), (1, False, True),
                                    (2, False, False), (2, False, True), (0, True, False), (0, True, True)):
        he.he_set_tuning(ctx, "ntt_generic", generic)
        he.he_set_tuning(ctx, "ntt_shape", shape)
        for _ in range(args.warmup):
            he.he_ntt(ctx, t, args.polys, nl * n, nl, 0, inverse)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(f"{'intt' if inverse else 'ntt'}_{'generic' if generic else f's{shape}'}")
        e0.record(stream)
        for _ in range(args.steps):
            he.he_ntt(ctx, t, args.polys, nl * n, nl, 0, inverse)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1) / args.steps
        limbs = args.polys * nl
        bfly = limbs * (n / 2) * log_n
        out[("intt" if inverse else "ntt") + ("_runtime_shaped" if generic else f"_shape{shape}" if shape else "")] = {
            "ms": ms, "Gbutterfly_s": bfly / ms / 1e6, "alu_frac": bfly / (ms * 1e-3) / ALU_PEAK["per_second"],
            "butterfly_chain_frac": bfly / (ms * 1e-3) / bfly_roof,
            "algorithmic_GBs_2pass": limbs * n * 32 / ms / 1e6 if log_n > 11 else limbs * n * 16 / ms / 1e6}
    he.he_set_tuning(ctx, "ntt_generic", False)
    print(json.dumps({"micro": "ntt", "N": n, "limbs": args.polys * nl, "steps": args.steps,
                      "butterfly_chain_per_s": bfly_roof, **out}))


def run_micro_keyswitch(args):
    """Rotation by 8 slots (automorphism + key switching) of `--polys`
    ciphertexts, with the per-class kernel times of the batch: at level 7 of
    the step's parameters (N = 2^14), or with --log-n 16 at the top level of
    the large parameters (24 x ~50-bit limbs, 4 special primes, dnum 6).
    --micro rotsum times one hoisted rotate-and-sum stage instead (rotations
    by 8, 16 and 24 sharing one decomposition).  --tune autotune runs the
    autotuner on this batch first."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_10091_gb300 as he
    measure_alu_peak(he)
    from paper_2006_10091_gb300 import workloads
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    hoisted = args.micro == "rotsum"
    steps = [8 * m for m in range(1, args.radix)] if hoisted else [8]
    if args.log_n == 16:
        ctx = he.Context(16, 24, 50, 4, 60, 2.0 ** 50, seed=0, rot_steps=steps, stream=stream.cuda_stream)
        level = 24
    else:
        ctx = he.Context(LOG_N, L, LIMB_BITS, ALPHA, SPECIAL_BITS, SCALE, seed=0, rot_steps=steps,
                         stream=stream.cuda_stream)
        level = L - 1

    def op(A, O):
        if hoisted:
            he.he_rotate_sum_batch(ctx, A, steps, O)
        else:
            he.he_rotate_batch(ctx, A, 8, O)
    count = args.polys
    tuned = None
    for kv in args.tune or []:
        if kv == "autotune":
            tuned = he.he_autotune(ctx, level, count)
            continue
        key, val = kv.split("=")
        he.he_set_tuning(ctx, key, float(val))
    host = workloads.residues(2, ctx.primes[:level], ctx.n, parts=2 * count).reshape(count, 2, level, ctx.n)
    A, O = ctx.new_ct(level, count), ctx.new_ct(level, count)
    he.he_ct_import_batch(ctx, host, level, ctx.scale, A)
    for _ in range(args.warmup):
        op(A, O)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        op(A, O)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    he.he_profile_enable(ctx, True)
    op(A, O)
    prof = {k: he.he_profile_read(ctx, k) for k in he.he_profile_names(ctx)}
    he.he_profile_enable(ctx, False)
    total_work = sum(v["work"] for v in prof.values())
    print(json.dumps({"micro": args.micro, "N": ctx.n, "level": level, "ciphertexts": count, "autotune": tuned,
                      "steps": steps, "ms_per_batch": ms, "rotations_per_s": len(steps) * count * 1000.0 / ms,
                      "modmul_per_s": total_work / (ms * 1e-3),
                      "alu_frac": total_work / (ms * 1e-3) / ALU_PEAK["per_second"],
                      "kernels": {k: {"ms": v["ms"], "GBs": v["bytes"] / max(v["ms"], 1e-9) / 1e6,
                                      "work_per_s": v["work"] / max(v["ms"], 1e-9) * 1e3}
                                  for k, v in prof.items()}}))


def run_micro_train(args):
    """Algorithms 1 and 2 as one loop (he_lr_train) at the step's parameters:
    K = 4 workers of 1024 samples x 784 features (128 data ciphertexts each),
    refresh (decrypt, average, re-encrypt) after every step (l = 1), `--steps`
    iterations timed; the decrypted weights against the same procedure in
    FP64."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_10091_gb300 as he
    from paper_2006_10091_gb300 import workloads
    from tests.lr_reference import lr_step_fp64
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n_slots = (1 << LOG_N) // 2
    ctx = he.Context(LOG_N, L, LIMB_BITS, ALPHA, SPECIAL_BITS, SCALE, seed=0, rot_steps=rot_steps(n_slots, G),
                     stream=stream.cuda_stream)
    he.he_autotune(ctx, L - 1, 64)
    coeffs = table2_binomial()
    K, ns = 4, 1024
    datas = [workloads.LRData(seed=500 + k, n_samples=ns, n_features=N_FEATURES) for k in range(K)]
    w0 = datas[0].w0
    lr = 1.0 / (K * ns)
    workers = []
    for k, d in enumerate(datas):
        zs = workloads.pack_samples(d.X, d.y, n_slots, G)
        Z = ctx.new_ct(L, len(zs))
        for i, v in enumerate(zs):
            he.he_encode_encrypt(ctx, v, SCALE, L, Z[i], cid=(k << 16) + i)
        W = ctx.new_ct(L)
        he.he_encode_encrypt(ctx, workloads.pack_weights(w0, n_slots, G), SCALE, L, W, cid=(k << 16) + 9999)
        workers.append((Z, W))
    cfg = he.lr_config(coeffs, lr, G, MASK_SCALE)
    out = ctx.new_ct(L)
    he.he_lr_train(ctx, workers, cfg, 1, 1, L, out)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    he.he_lr_train(ctx, workers, cfg, args.steps, 1, L, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ws = [w0.copy() for _ in datas]
    for _ in range(args.steps):
        ws = [lr_step_fp64(d.X, d.y, w, coeffs, lr) for d, w in zip(datas, ws)]
        avg = sum(ws) / len(ws)
        ws = [avg.copy() for _ in ws]
    want = workloads.pack_weights(ws[0], n_slots, G)
    got = he.he_decrypt_decode(ctx, out)
    print(json.dumps({"micro": "train", "workers": K, "samples_per_worker": ns, "features": N_FEATURES,
                      "refresh_every": 1, "iterations": args.steps, "ms": ms,
                      "iterations_per_s": args.steps * 1000.0 / ms,
                      "worker_steps_per_s": K * args.steps * 1000.0 / ms,
                      "max_rel_err_vs_fp64": float(np.max(np.abs(got - want)) / np.max(np.abs(want)))}))


def run_part(args):
    """One of the extra measurements alone (batched workers or serving)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_10091_gb300 as he
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.micro == "workers":
        print(json.dumps({"part": "batched_workers", **batched_workers(he, torch, stream)}))
    else:
        print(json.dumps({"part": "serving", **serving(he, torch, stream, n_requests=args.requests,
                                                       inflight=args.serve_inflight, wave=args.serve_wave)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--micro", choices=["ntt", "keyswitch", "rotsum", "workers", "serving", "alu", "train"],
                    default=None,
                    help="time one kernel class or one extra measurement alone")
    ap.add_argument("--requests", type=int, default=400, help="timed requests of --micro serving")
    ap.add_argument("--tune", action="append", help="key=value tuning knob (he_set_tuning) applied after the autotuner")
    ap.add_argument("--serve-inflight", type=int, default=4, help="waves per context in --micro serving")
    ap.add_argument("--serve-wave", type=int, default=16, help="requests per wave in --micro serving")
    ap.add_argument("--log-n", type=int, default=14)
    ap.add_argument("--radix", type=int, default=4, help="--micro rotsum: rotations by 8, 16, ..., 8*(radix-1)")
    ap.add_argument("--polys", type=int, default=256)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the extra multiplication-rate lines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chunk-bytes", type=float, default=float(1 << 35),
                    help="scratch budget of one batched operation (default 32 GiB: the step's 512 data "
                         "ciphertexts in one batch)")
    ap.add_argument("--graph", action="store_true", help="replay the step as a captured CUDA graph")
    ap.add_argument("--alpha", type=int, default=None, help="special primes of the step's parameters")
    ap.add_argument("--special-bits", type=int, default=None)
    args = ap.parse_args()
    global ALPHA, SPECIAL_BITS
    if args.alpha is not None:
        ALPHA = args.alpha
    if args.special_bits is not None:
        SPECIAL_BITS = args.special_bits
    if args.micro == "ntt":
        run_micro(args)
        return
    if args.micro in ("keyswitch", "rotsum"):
        run_micro_keyswitch(args)
        return
    if args.micro == "train":
        run_micro_train(args)
        return
    if args.micro in ("workers", "serving"):
        run_part(args)
        return
    if args.micro == "alu":
        import __graft_entry__
        __graft_entry__.build()
        import paper_2006_10091_gb300 as he
        names = ("imad_32", "shoup_product_64", "lazy_butterfly_radix8", "mac_128", "mac_split3")
        print(json.dumps({"micro": "alu", **{n: he.he_probe_alu(k) for k, n in enumerate(names)},
                          "fallback_roof": {"per_second": ALU_MODMUL_PEAK,
                                            "note": "152 SMs x 2070 MHz x 64 / 17.3 (Shoup product)"}}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
