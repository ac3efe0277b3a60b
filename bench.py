#!/usr/bin/env python
"""Throughput of the FB expansion + steerable covariance hot path (Alg. 1 steps
3-4 and Alg. 2 steps 1-4 accumulation) at L = 128 on GB300.

One step = ffb_expand + ffb_covariance(reset) over the whole stack of
n = 100000 synthetic Gaussian-blob images (L = 128, R = 64, c = 1/2,
SNR = 1/10; 6.55 GB, larger than L2, resident in HBM before timing).
Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the same workload instead (a bounded sample per step).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "images/sec FB expansion+covariance at L=128 (compensated TC vs FP32), % roofline"
UNIT = "images/s"
L_, C_, R_, EPS = 128, 0.5, 64.0, 1e-6


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", help="fp32|bf16|bf16x3|tf32|tf32x3|auto")
    ap.add_argument("--n", type=int, default=0, help="override images per GPU (testing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-post", action="store_true", help="skip the a8-a10 timings after the step")
    ap.add_argument("--no-batching", action="store_true", help="skip the 48-stack batching workload after the step")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic work per image (flops) of each kernel class, and its roofline
# ---------------------------------------------------------------------------
def algorithmic_flops(plan, eps=EPS):
    """Algorithmic flops per image of each kernel class: the work the method
    needs, counted as the scope table of the hot path counts it (5 n log2 n
    per complex FFT of length n, half of it for a real-input or Hermitian
    transform; 2 flop per real multiply-add).

    * interpolation: n_xi * n_theta/2 half-polar nodes x w_a^2 taps x 5 flop
      (4 for the complex value times a real weight, 1 for the separable weight
      product), w_a = ceil(log10(1/eps)) + 1 the width the accuracy needs
      (the kernel runs w_a + 1 = 8 taps, see ``executed_flops``);
    * oversampled 2-D FFT: real input, half of whose rows are zero padding:
      2.5 N^2 log2(N^2) / 2;
    * ring DFT: each ring is Hermitian (F(theta + pi) = conj F(theta)), so a
      real-input count 2.5 n_theta log2 n_theta per ring;
    * radial quadrature: 4 P n_xi (complex vector times real matrix);
    * covariance: 2 sum_k p_k^2 (real SYRK of the Re and Im parts, symmetric
      half)."""
    n_xi, nth, N = plan.n_xi, plan.n_theta, plan.N
    w_a = math.ceil(math.log10(1.0 / eps) - 1e-12) + 1
    interp = n_xi * (nth // 2) * w_a * w_a * 5
    fft2 = 2.5 * N * N * math.log2(N * N) / 2
    ring = n_xi * 2.5 * nth * math.log2(nth)
    return {
        "interp_ring": fft2 + interp + ring,   # separate-kernel path (rows, cols, interp + ring kernels)
        "rows_fft": fft2 / 2,                  # L real rows of length N: half of the 2-D count
        "cols_fft": fft2 / 2,
        "grid_interp": fft2 + interp,          # shared-memory grid path
        "ring_fft": ring,
        "bessel": 4.0 * plan.P * n_xi,
        "covariance": 2.0 * sum(pk * pk for pk in plan.p),
    }


def executed_flops(plan):
    """Flops per image that the kernels execute (context for the
    algorithmic counts above): w = plan.w taps of 4 flop per half-polar node,
    complex FFTs of every row pair and of the N/2 + 1 column half, full
    complex ring FFTs of length n_theta."""
    n_xi, nth, w, N, L = plan.n_xi, plan.n_theta, plan.w, plan.N, plan.L
    fftN = 5 * N * math.log2(N)
    return {"grid_interp": (L / 2) * fftN + (N / 2 + 1) * fftN + n_xi * (nth // 2) * w * w * 4,
            "ring_fft": n_xi * 5 * nth * math.log2(nth)}


def tc_ring_dft(plan, precision):
    """Whether the plan's ring DFT runs as the dense tensor-core contraction
    (BF16x3, shared-memory grid path, n_theta = 512, 128 rings), and its
    executed flops per image: two parities x three products x 128 rings x
    192 table columns x 256 samples x 2."""
    on = precision == "bf16x3" and plan.polar_variant > 0 and plan.n_theta == 512 and plan.n_xi == 128
    return on, (2 * 3 * plan.n_xi * 192 * (plan.n_theta // 2) * 2 if on else 0)


PROF_STRIDE = 32   # kernel timing: every 32nd launch of each kernel class
POST_N = 20000     # images for the a8-a10 timings after the step


def hbm_floor(plan):
    """images/s if only the image in (L^2 float32) and the coefficients out
    (P complex float32) crossed HBM, at the measured copy bandwidth."""
    try:
        gbs = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        gbs = 6800.0
    return gbs * 1e9 / (plan.L * plan.L * 4 + plan.P * 8)


# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of a 152-image launch (the committed profile of the four-node-unit
# grid kernel at L = 128), valid only
# while the kernel's sources are byte-identical to the profiled ones (the
# kernel's file from its top through the kernel, i.e. its macros, device
# helpers and body, and the register-FFT header; from ffb_internal.cuh it uses
# only the complex arithmetic and the status flag).  ncu empties L2 before the
# capture, so the figure includes one read of the plan's 3 MB unit table,
# which stays in L2 between launches in a live run.
NCU_TRAFFIC = {
    "grid_interp": {"sources": ["paper_1412_0781_gb300/csrc/ffb_grid.cu:^k_grid_interp_half",
                                "paper_1412_0781_gb300/csrc/ffb_fft.cuh"],
                    "sha256": "7c1b52d63320b99dafa946b70647e582c41079b925af4f2d76dd0b0ccd0abc12",
                    "bytes_per_launch": 17974784 + 54528, "images_per_launch": 152},
}


def _source_digest(sources):
    """sha256 over the listed files (the kernel's file and the header its
    inlined helpers come from); "file:kernel" hashes only the text from the
    kernel's template line to the next section banner, "file:^kernel" the
    text from the top of the file (its macros and device helpers) to that
    banner, so that host code further down does not count."""
    import hashlib
    h = hashlib.sha256()
    for src in sources:
        path, _, kern = src.partition(":")
        txt = open(os.path.join(ROOT, path)).read()
        if kern:
            top = kern.startswith("^")
            kern = kern.lstrip("^")
            a = txt.index(kern + "(")
            a = txt.rindex("template", 0, a)
            b = txt.index("\n// " + "-" * 75 + "\n", a)   # the next full-width section banner
            txt = txt[:b] if top else txt[a:b]
        h.update(txt.encode())
    return h.hexdigest()


def ncu_traffic(kernel, images_per_launch):
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None or _source_digest(rec["sources"]) != rec["sha256"]:
        return None
    return rec["bytes_per_launch"] * images_per_launch / rec["images_per_launch"]


def measured_tensor_peak(precision):
    """Sustained dense tensor-core peak for the contraction's input type, from
    MEASURED_PEAKS.json (bf16 measured; tf32 by the nominal 1.1 / 2.25 ratio);
    the recipe's 1.7 PFLOP/s sustained figure when the file is absent."""
    if precision not in ("bf16", "bf16x3", "tf32", "tf32x3"):
        return None, None
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bf16, src = float(pk["bf16_tflops_sustained"]), "of measured sustained bf16"
    except (OSError, KeyError, ValueError):
        bf16, src = 1700.0, "of fallback sustained bf16"
    if precision.startswith("tf32"):
        return bf16 * 1.1 / 2.25, src + " x 1.1/2.25 (tf32)"
    return bf16, src


def fp32_peak_tflops(sms, sm_mhz):
    """SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# the batching workload after the step: 48 stacks of uneven L and n
# ---------------------------------------------------------------------------
def batching_run(dev, precision, reps=3):
    """a1-a7 over the 48-stack batching workload (L in {64, 96, 128, 180, 256},
    n in [500, 20000], about 53 GB of images resident in HBM) through one
    group call per step: per-stack expansion branches, one grouped covariance
    launch, a CUDA graph replayed after the eager and the capturing call.
    Returns images/s over ``reps`` replays timed with CUDA events."""
    import torch
    from paper_1412_0781_gb300 import Group, Plan, data
    specs = data.batching_stacks()
    plans = [Plan(sp.L, sp.c, sp.R, eps=EPS, precision=precision) for sp in specs]
    imgs = [data.blob_stack(sp, device=dev)[0] for sp in specs]
    coefs = [torch.empty((sp.n, p.P, 2), device=dev, dtype=torch.float32) for sp, p in zip(specs, plans)]
    g = Group(plans)
    t0 = time.perf_counter()
    g.expand_cov(imgs, coefs, reset=True)          # eager call (tunes the grouped covariance once)
    g.sync()
    eager_s = time.perf_counter() - t0
    g.expand_cov(imgs, coefs, reset=True)          # captures the CUDA graph
    g.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        g.expand_cov(imgs, coefs, reset=True)      # graph replays
    b.record()
    torch.cuda.synchronize()
    g.sync()
    ms = a.elapsed_time(b) / reps
    n_img = sum(sp.n for sp in specs)
    img_bytes = sum(sp.n * sp.L * sp.L * 4 for sp in specs)
    by_L = {}
    for sp in specs:
        by_L.setdefault(sp.L, [0, 0])
        by_L[sp.L][0] += 1
        by_L[sp.L][1] += sp.n
    info = g.info()
    out = {"stacks": len(specs), "images": n_img, "image_bytes": img_bytes,
           "coef_bytes": sum(sp.n * p.P * 8 for sp, p in zip(specs, plans)),
           "stacks_and_images_by_L": {str(k): v for k, v in sorted(by_L.items())},
           "precision": precision, "ms_per_call": ms, "images_per_s": n_img / (ms / 1e3),
           "eager_call_s": eager_s, "graph_replays_timed": reps,
           "grouped_covariance_item": {"images_per_item": info["per"], "tile": info["tile"], "grid": info["grid"],
                                       "candidates_timed": info["candidates"]},
           "launches_per_call": info["launches"],
           "note": "a1-a7 of every stack in one group call (expansion branches, one grouped covariance launch), "
                   "replayed CUDA graph; inputs resident in HBM"}
    g.close()
    for p in plans:
        p.close()
    del imgs, coefs
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def oracle_rate(budget_s=15.0, max_images=1024):
    """FP64 oracle (direct NDFT, plain ring DFT, quadrature, two-pass
    covariance) on a bounded sample of the L = 128 workload, images/s."""
    import numpy as np
    from oracle import fb
    from paper_1412_0781_gb300 import data
    op = fb.make_plan(L_, C_, R_)           # precomputation, untimed
    imgs, _, _ = data.blob_stack(data.PRECISION_L128, n=max_images)
    x = imgs.double().numpy()
    fb.expand(op, x[:1])                    # warm the cached NDFT factors
    t0 = time.perf_counter()
    done = 0
    while done < max_images and (time.perf_counter() - t0) < budget_s:
        a = fb.expand(op, x[done:done + 4])
        fb.covariance(op, a)
        done += a.shape[0]
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    rates = []
    for _ in range(args.warmup):
        oracle_rate(budget_s=2.0, max_images=4)
    total_imgs, total_t = 0, 0.0
    for _ in range(args.steps):
        r, m, dt = oracle_rate(budget_s=max(2.0, 60.0 / max(1, args.steps)), max_images=16)
        rates.append(r)
        total_imgs += m
        total_t += dt
    value = total_imgs / total_t
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "precision stack L=128 R=64 c=0.5 SNR=1/10 (n=100000)", "L": L_,
                       "n": 100000, "oracle_sample_images": total_imgs},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d images of the n=100000 L=128 stack per run, direct NDFT" % total_imgs},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1412_0781_gb300 import Plan, data

    spec = data.PRECISION_L128
    n = args.n or spec.n
    images, _, sigma2 = data.blob_stack(data.StackSpec(n, spec.L, spec.R, spec.n_blobs, spec.width, spec.snr,
                                                  spec.seed + 7919 * rank), device=dev)
    if args.precision == "auto":
        precisions = ["fp32", "tf32x3", "bf16x3", "tf32", "bf16"]
    else:
        precisions = [args.precision]
    results = {}
    coef = None
    for prec in precisions:
        plan = Plan(L_, C_, R_, eps=EPS, precision=prec)
        if coef is None:
            coef = torch.empty((n, plan.P, 2), device=dev, dtype=torch.float32)

        def step():
            plan.expand(images, out=coef)
            plan.covariance(coef, reset=True)

        for _ in range(max(3, args.warmup)):
            step()
        plan.sync()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = plan.launch_count()
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        # kernel durations from CUDA events around every PROF_STRIDE-th launch
        # of each kernel class inside the timed region (events around every
        # launch would add their own cost to the step)
        plan.profile(True, stride=PROF_STRIDE)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        prof = plan.profile_read()
        plan.profile(False)
        plan.sync()
        launches = plan.launch_count() - l0
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        results[prec] = {"plan": plan, "coef": coef, "ms": ms, "prof": prof, "clocks": clocks,
                         "launches": launches}
    # headline: the faster compensated tensor-core form (both gated at 1e-5
    # against the FP64 oracle in tests/test_gpu_tc.py); else the one run
    comp = [p for p in ("tf32x3", "bf16x3") if p in results]
    head = min(comp, key=lambda p: results[p]["ms"]) if comp else precisions[0]
    for p, v in results.items():
        if p != head:
            v["plan"].close()
    r = results[head]
    plan = r["plan"]
    ms_step = r["ms"] / args.steps
    value = world * n / (ms_step / 1e3)

    # roofline of the dominant kernel (largest share of the timed region)
    flops = algorithmic_flops(plan)
    prof = r["prof"]
    dom = max(prof, key=lambda c: prof[c][0])
    dom_ms, dom_calls = prof[dom]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (r["clocks"] or {}).get("sm_max_mhz") or 2070.0
    share = {c: round(v[0] / sum(x[0] for x in prof.values()), 4) for c, v in prof.items()}
    imgs_per_launch = (n * args.steps) / dom_calls if dom_calls else 0
    achieved = flops.get(dom, 0.0) * imgs_per_launch / (dom_ms / dom_calls / 1e3) / 1e12 if dom_calls else 0.0
    peak = fp32_peak_tflops(sms, max_mhz)
    exe = executed_flops(plan)
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dom, imgs_per_launch),
                "algorithmic_mflop_per_image": flops.get(dom, 0.0) / 1e6,
                "executed_mflop_per_image": exe.get(dom, 0.0) / 1e6,
                "peak_note": "FP32 FFMA peak %d SMs x 128 lanes x 2 flop x %.0f MHz (derived, max clock)" % (
                    sms, max_mhz),
                "kernel_ms_per_launch": dom_ms / dom_calls, "images_per_launch": imgs_per_launch,
                "kernel_timing": "CUDA events around every %dth launch of each kernel in the timed region" % PROF_STRIDE,
                "share": share}

    # the whole step against its floor: the FP32-ALU work of a1-a4 at the
    # FFMA peak (the tensor-core and HBM floors are far higher)
    tc_ring, _ = tc_ring_dft(plan, head)
    alu_flops = flops["grid_interp"] + (0.0 if tc_ring else flops["ring_fft"])
    floor = peak * 1e12 / alu_flops
    roofline["step"] = {"bound": "alu", "floor_images_per_s": floor, "frac": value / floor,
                        "note": "%s FP32 work %.2f MFLOP/image at the FFMA peak; HBM floor %.1f M images/s" % (
                            "a1-a3 (the ring DFT runs on the tensor cores)" if tc_ring else "a1-a4",
                            alu_flops / 1e6, hbm_floor(plan) / 1e6)}

    # end to end through the public API with host buffers, right after the
    # timed step (the same plan, before the after-step timings)
    e2e = None
    if not args.no_e2e and rank == 0:
        hbuf = torch.empty(images.shape, dtype=torch.float32, pin_memory=True)
        hbuf.copy_(images)
        out_mean = torch.empty(plan.p[0], dtype=torch.float64, pin_memory=True)
        out_C = torch.empty(plan.cov_total, dtype=torch.float64, pin_memory=True)

        def e2e_step():
            # one C-ABI call: host images in, host mean and covariance out; the
            # library copies the images in parts on its own stream, each part
            # overlapping the expansion of the one before
            plan.expand_cov_host(hbuf, reset=True, mean_out=out_mean, C_out=out_C)

        def h2d_rate():
            # one plain copy of the whole pinned buffer: the host link's rate
            # at the time (it is shared with other tenants of the machine)
            dtmp = torch.empty(hbuf.shape, dtype=torch.float32, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dtmp.copy_(hbuf, non_blocking=True)
            torch.cuda.synchronize()
            rate = hbuf.numel() * 4 / (time.perf_counter() - t0) / 1e9
            del dtmp
            torch.cuda.empty_cache()
            return rate

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        h2d_before = h2d_rate()
        # host clock around every step (each ends with the covariance on the
        # host); the value is total images / total time over k steps
        k = max(5, args.steps // 2)
        steps_ms = []
        e2e_clk = ClockSampler(local)
        e2e_clk.start()
        time.sleep(0.3)
        for _ in range(k):
            ts = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            steps_ms.append((time.perf_counter() - ts) * 1e3)
        e2e_clocks = e2e_clk.stop()
        dt = sum(steps_ms) / 1e3 / k
        e2e = {"value": n / dt, "unit": UNIT, "h2d_bytes_per_step": int(hbuf.numel() * 4),
               "d2h_bytes_per_step": int((plan.p[0] + plan.cov_total) * 8), "steps": k,
               "median_step_ms": statistics.median(steps_ms), "max_step_ms": max(steps_ms),
               "call": "ffb_expand_cov_host (pinned host images -> host mean and covariance)",
               "h2d_gbs_plain_copy": [round(h2d_before, 1), round(h2d_rate(), 1)], "clocks": e2e_clocks}
        del hbuf

    # a8-a10 after the timed step (reported beside the metric, not part of
    # it): the eigendecomposition of the step's covariance, MP-Wiener
    # denoising (a9 selection and filter, a10 synthesis through the adjoint,
    # including the images' own expansion) and the adjoint alone, on the first
    # POST_N images, each timed with CUDA events after one untimed run
    post = None
    if rank == 0 and not args.no_post:
        m = min(n, POST_N)
        sub = images[:m]

        def timed(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        eig_ms = timed(lambda: plan.eig())
        den = torch.empty_like(sub)
        den_ms = timed(lambda: plan.denoise(sub, mode="mp_wiener", sigma2=sigma2, out=den))
        adj = torch.empty_like(sub)
        adj_ms = timed(lambda: plan.expand_adjoint(r["coef"][:m], out=adj))
        # the rows beyond the hot path: radial eigenfunctions and the top-20
        # eigenimages, the SVD route and the rotation-invariant features on
        # the first m coefficients (with the HBM share of their coefficient
        # reads), R and c from the first m images
        ev, _ = plan.eig()
        evn = ev.cpu().numpy()
        offs = list(plan.offset) + [plan.P]
        top = sorted(range(plan.P), key=lambda t: -evn[t])[:20]
        pairs = []
        for t in top:
            k = max(i for i in range(plan.k_max + 1) if offs[i] <= t)
            pairs.append((k, t - offs[k]))
        f1_rad_ms = timed(lambda: plan.radial_eigenfunctions())
        f1_img_ms = timed(lambda: plan.eigenimages(pairs))
        coef_m = r["coef"][:m]
        coef_bytes = m * plan.P * 8
        f2_svd_ms = timed(lambda: plan.svd(coef_m))
        inv_pairs = pairs[:10]
        triples = [(1, 0, 1, 0, 0), (1, 0, 2, 0, 0), (2, 0, 1, 0, 0), (1, 0, 0, 0, 0)]
        f2_inv_ms = timed(lambda: plan.invariants(coef_m, inv_pairs, triples))
        f3_est_ms = timed(lambda: plan.estimate_support(sub), reps=1)
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        post = {"a8_eig_ms": eig_ms, "eig_blocks": plan.k_max + 1,
                "a9_a10_denoise_images_per_s": m / (den_ms / 1e3), "a10_adjoint_images_per_s": m / (adj_ms / 1e3),
                "images": m, "mode": "mp_wiener (known noise variance)",
                "next1_radial_eigenfunctions_ms": f1_rad_ms, "next1_eigenimages_20_ms": f1_img_ms,
                "next2_svd_route_ms": f2_svd_ms,
                "next2_svd_coef_read_frac_hbm": coef_bytes / (f2_svd_ms / 1e3) / (hbm * 1e9),
                "next2_invariants_images_per_s": m / (f2_inv_ms / 1e3),
                "next2_invariants_coef_read_frac_hbm": coef_bytes / (f2_inv_ms / 1e3) / (hbm * 1e9),
                "next3_estimate_support_images_per_s": m / (f3_est_ms / 1e3)}
        del den, adj

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        rate, m, dt = oracle_rate()
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d images of the n=100000 L=128 stack (%.1f s), FP64 direct NDFT + ring DFT + "
                         "quadrature + covariance; numpy BLAS threads" % (m, dt)}

    if post is not None and not args.no_batching:
        r["coef"] = coef = None
        torch.cuda.empty_cache()
        post["batching"] = batching_run(dev, head)

    # every stage against its own roof: the FFT / NUFFT stages against the FP32
    # FFMA peak, the contractions against the tensor-core peak of their input
    # type (measured sustained bf16; tf32 = bf16 x 1.1/2.25, the nominal ratio)
    stages = {}
    tc_peak, tc_note = measured_tensor_peak(head)
    for c, (ms_c, calls_c) in prof.items():
        if c not in flops or ms_c <= 0:
            continue
        rate = flops[c] * n * args.steps / (ms_c / 1e3) / 1e12
        contraction = c in ("bessel", "covariance")
        tc_ring, ring_exec = tc_ring_dft(plan, head)
        if c == "ring_fft" and tc_ring and tc_peak:
            exe_rate = ring_exec * n * args.steps / (ms_c / 1e3) / 1e12
            stages[c] = {"bound": "tensor", "achieved": rate, "executed": exe_rate, "peak": tc_peak,
                         "unit": "TFLOP/s", "frac": exe_rate / tc_peak, "peak_note": tc_note,
                         "ms_per_step": ms_c / args.steps,
                         "note": "dense ring DFT on the tensor cores, %.1f MFLOP/image executed (BF16x3); "
                                 "achieved counts the FFT's %.2f MFLOP/image" % (ring_exec / 1e6, flops[c] / 1e6)}
        elif contraction and tc_peak:
            products = 3 if head in ("bf16x3", "tf32x3") else 1
            stages[c] = {"bound": "tensor", "achieved": rate, "executed": rate * products, "peak": tc_peak,
                         "unit": "TFLOP/s", "frac": rate * products / tc_peak, "peak_note": tc_note,
                         "ms_per_step": ms_c / args.steps}
        else:
            stages[c] = {"bound": "alu", "achieved": rate, "peak": peak, "unit": "TFLOP/s", "frac": rate / peak,
                         "ms_per_step": ms_c / args.steps}
            if c == "grid_interp" and plan.polar_variant > 0:
                # what the interpolation moves through the L1 / shared-memory
                # pipe: per unit of the plan's table, the 9 x 9 union of
                # complex grid values (81 gathers of 8 bytes) and its record
                # (19 float4 = 304 bytes), counted from the table itself
                from paper_1412_0781_gb300 import ffb as ffb_mod
                import numpy as np
                _, xi_t, _, _ = plan.tables()
                rec, _, _, _, _, _ = ffb_mod.interp_units(plan.N, plan.w, 2.30 * plan.w, plan.n_theta, xi_t)
                units = int(np.count_nonzero((rec[:, 18, :, 1].copy().view(np.uint32) & 0xFFFF) != 0xFFFF))
                l1_bytes = units * (81 * 8 + 19 * 16)
                l1_rate = l1_bytes * n * args.steps / (ms_c / 1e3) / 1e12
                l1_peak = sms * 128 * max_mhz * 1e6 / 1e12
                stages[c]["l1"] = {"achieved": l1_rate, "peak": l1_peak, "unit": "TB/s", "frac": l1_rate / l1_peak,
                                   "bytes_per_image": l1_bytes,
                                   "units_per_image": units,
                                   "note": "interpolation gathers + unit records through L1 / shared memory; peak "
                                           "%d SMs x 128 B/clk x %.0f MHz (derived); the FFT phases add more" % (
                                               sms, max_mhz)}

    if rank == 0:
        # the comparison the metric names, up front: the same step in FP32
        fp32 = None
        if "fp32" in results and head != "fp32":
            v32 = world * n / (results["fp32"]["ms"] / args.steps / 1e3)
            fp32 = {"value": v32, "speedup": value / v32}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "vs_fp32": fp32, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "tf32x3": "tf32x3 (f32 acc)", "bf16x3": "bf16x3 (f32 acc)",
                                                "tf32": "tf32", "bf16": "bf16"}[head],
                "data": "synthetic",
                "config": {"workload": "precision stack: n=100000 Gaussian-blob images L=128 R=64 c=0.5 "
                                       "SNR=1/10, eps=1e-6", "L": L_, "n_per_gpu": n, "precision": head,
                           "l2": "inputs (6.55 GB) larger than L2, no flush",
                           "polar_variant": {0: "separate grid and interpolation kernels", 1: "grid in shared memory",
                                             2: "grid in shared memory, CTA-pair clusters"}[r["plan"].polar_variant]},
                "precisions": {p: {"images_per_s": world * n / (v["ms"] / args.steps / 1e3),
                                   "kernel_ms": {c: round(t[0] / args.steps, 4) for c, t in v["prof"].items()}}
                               for p, v in results.items()},
                "roofline": roofline, "stages": stages, "after_step": post, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": r["launches"],
                "clocks": r["clocks"]}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
