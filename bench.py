"""Benchmark: planet-observation evaluations per second of the batched
Keplerian radial-velocity chi-square (mixed precision vs FP64) on GB300.

Workload (default): the paper-shaped batch, n_sys = 4096 model systems with
n_pl = 4 planets against n_obs = 256 observations of one star (synthetic,
seeded; the paper's data set is not available).  One step = one fused
chi-square evaluation of the whole batch (mean anomaly, Kepler solve,
velocities, residuals, per-system reduction) through the C ABI.

Timing: W warm-up steps, then K timed steps bracketed by a barrier and
device synchronisation.  The K steps run back to back between one pair of
CUDA events on the launching stream, each on its own copy of the inputs
from a rotating pool larger than L2 (256 MiB), so that no step finds its
inputs in L2 and nothing is flushed.  Beside it the line reports the same
steps each between its own CUDA events with L2 flushed before it: a
256 MiB buffer is written and then a second one read, so every step starts
with a cold L2 holding no dirty lines (otherwise the write-back of the
flush buffer lands inside the next timed kernel).  Multi-GPU (torchrun): every
rank evaluates its own batch of the same shape (weak scaling, no
data-path collective); the slowest rank's time is reported.

`--impl reference` times the FP64 CPU oracle instead (the paper's
CPU-reference role), on the host cores, on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# the headline metric; both arms (this library and the oracle) report it
METRIC_PAPER_BATCH = "planet-obs evals/s (chi2, npl=4, nobs=256) mixed vs FP64"
FP32_LANES_PER_SM = 128
# the rotating pool of timed inputs spans this many bytes (twice the L2)
ROTATE_BYTES = 256 << 20
FALLBACK_SM_MHZ = 2070.0

# Algorithmic FP32 work of one planet-observation evaluation of the mixed
# path, in FLOPs (FMA = 2, add/mul = 1; MUFU sin/cos/rcp and integer or
# select operations not counted), from the algorithm as implemented:
#   double-single mean anomaly 18 (its low part formed already scaled by
#   2 pi), Mikkola's starting value 18 (its per-planet constants and the
#   MUFU square root, logarithm, exponential and reciprocals not counted),
#   one accurate sin/cos 27, the Halley step 11, sin/cos update of the step
#   10, velocity 8, planet Kahan sum 4, and per observation the residual +
#   weighted square + chi2 Kahan sum 10 (shared by n_pl planets).  The
#   per-(system, planet) setup is not counted.
KEPLER_MIXED_FLOPS = 18 + 27 + 11 + 10
MEAN_ANOMALY_FLOPS = 18


def mixed_flops_per_eval(n_pl: int, warp: bool = False) -> float:
    """FLOPs per evaluation of the mixed chi2 kernels (the tile kernels and
    the warp-per-system kernel run the same per-evaluation arithmetic)."""
    return MEAN_ANOMALY_FLOPS + KEPLER_MIXED_FLOPS + 8 + 4 + 10.0 / n_pl


def mixed_kernel_name(n_pl: int, tile) -> str:
    return (f"chi2_mixed_warp_kernel<{n_pl}>" if tile[2] == 3 else
            f"chi2_mixed_kernel<{n_pl}>")


# The adjoint adds, per planet and observation: the velocity partials 26
# (cos f, sin f, cos/sin(w + f), dK, dw, dM, de), 1/D 2, dP 3, the
# compensated dP sum 5 and the four other accumulations 8; per observation
# the weighted residual, chi2 sum and gamma term 12 (instead of 10).
def grad_flops_per_eval(n_pl: int) -> float:
    return MEAN_ANOMALY_FLOPS + KEPLER_MIXED_FLOPS + 8 + 4 + 44 + 12.0 / n_pl


# The Gauss-Newton pass adds the row u = sqrt(w) J of U (5 products per
# planet, 1 per observation) on the FP32 pipe; its U^T U update runs on the
# tensor cores (reported separately).
def gn_flops_per_eval(n_pl: int) -> float:
    return grad_flops_per_eval(n_pl) + 5 + 1.0 / n_pl


def gn_tensor_flops_per_obs(n_pl: int, split: int) -> float:
    """Tensor FLOPs per (system, observation) of the U^T U update as issued
    (2 FLOP/MAC).  split 0 (mma.sync): 16 x 8 x 8 tiles on or above the
    diagonal, three TF32 products each.  split 4 (tcgen05): M = N = 64 tiles
    shared by four systems, two TF32 products (hi hi^T, lo hi^T)."""
    if split == 4:
        return 2 * 64 * 64 * 2 / 4
    n = 5 * n_pl + 1
    mt, nt = (n + 15) // 16, (n + 7) // 8
    tiles = sum(1 for m in range(mt) for q in range(nt) if 8 * q + 7 >= 16 * m)
    return tiles * 3 * 16 * 8 * 2          # per observation (K = 1 of each 8-deep step)


# FP64 path, FP64 FLOPs per planet-observation evaluation (FMA = 2), from its
# algorithm: mean anomaly 6 (tau/P minus its integer part in one FMA, the
# offset, the removal of the nearest integer, the scaled FMA; the integer
# parts and the low part of the phase in single precision), table-driven
# sin/cos 20 (reduction 4, b^2 and b^3 2, sin b to b^3 2, cos b to b^4 4,
# table combination 8; the b^5 and b^6 terms in single precision), Halley
# step with a one-Newton-step reciprocal 13, last-step update 8, velocity
# with a one-Newton-step reciprocal and the planet sum's addition 11 (the
# FP32 presolve, the single-precision correction terms and reciprocal seeds
# and the per-CTA table are not counted).
F64_FLOPS_PER_EVAL = 6 + 20 + 13 + 8 + 11


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the mixed chi2 kernel in its current form, from ncu captures of this
# benchmark's own default workload at the two tiles its autotuner picks
# (the warp-per-system kernel with 27- or 28-warp CTAs, within 0.1 % of each
# other back to back): the batch reads its 688 KB of parameters and 6 KB of
# observations once (the rest is sector granularity of the 168-byte
# parameter rows).  Keyed by (config, n_sys override, tile); other launches
# report null.
DRAM_BYTES_PER_LAUNCH = {(1, None, (32, 864, 3)): 763904, (1, None, (32, 896, 3)): 763904}


def sm_count() -> int:
    """SMs of the current CUDA device (queried, not assumed)."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def sm_mhz_for_peaks():
    pk, _ = peaks()
    return pk.get("sm_max_mhz", FALLBACK_SM_MHZ)


def hold_gpu(stream, host_us):
    """Queue a bounded spin of the GPU clock (torch.cuda._sleep, a fixed
    cycle count) ahead of a timed loop, long enough for the host to enqueue
    the whole loop meanwhile: the GPU then reaches every start event with
    the step's work already queued, so the CUDA events bracket GPU work, not
    host-side launch latency (or a host stalled by the clock sampler)."""
    import torch
    sleep = getattr(torch.cuda, "_sleep", None)
    if sleep is None:            # not in this torch build: time without the hold
        return
    cycles = int(max(2000.0, host_us) * sm_mhz_for_peaks())
    with torch.cuda.stream(stream):
        sleep(cycles)


def kepler_throughput(kc, dev, stream, n=1 << 24):
    """Solutions of Kepler's equation per second (the paper's Table 2 also
    reports this), FP32 and FP64, on n random (M, e) pairs, e <= 0.95."""
    import torch
    g = torch.Generator(device=dev).manual_seed(7)
    M = (torch.rand(n, device=dev, generator=g, dtype=torch.float64) * 2 - 1) * 3.141592653589793
    e = torch.rand(n, device=dev, generator=g, dtype=torch.float64) * 0.95
    out = {}
    for mode, Mx, ex in (("mixed", M.float(), e.float()), ("fp64", M, e)):
        E = torch.empty_like(Mx)
        for _ in range(3):
            kc.kc_kepler_solve(Mx, ex, mode=mode, out=E, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hold_gpu(stream, 10 * 200.0)
        a.record(stream)
        for _ in range(10):
            kc.kc_kepler_solve(Mx, ex, mode=mode, out=E, stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        out["fp32" if mode == "mixed" else "fp64"] = 10 * n / (a.elapsed_time(b) / 1e3)
    out["unit"] = "Kepler solutions/s"
    return out


def oracle_subset(w, n_sub, grad=False):
    """The FP64 oracle on n_sub evenly spaced systems of a uniform workload,
    on the host cores (OpenMP over systems); planet-obs evals/s of chi2 (and
    its gradient with grad).  Its observations are formed by the oracle
    from the same seeded draws."""
    import oracle
    oracle.build()
    v = oracle.predict(w.truth, w.t, w.n_pl, w.t0)[0] + w.noise
    idx = np.unique(np.linspace(0, w.n_sys - 1, n_sub).astype(np.int64))
    par = np.ascontiguousarray(w.params[idx])
    oracle.chi2(par[:16], w.t, v, w.sigma, w.n_pl, w.t0, grad=grad)          # warm
    t_start = time.perf_counter()
    oracle.chi2(par, w.t, v, w.sigma, w.n_pl, w.t0, grad=grad)
    el = time.perf_counter() - t_start
    return {"value": idx.size * w.n_pl * w.n_obs / el, "unit": "planet-obs evals/s",
            "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{idx.size} evenly spaced systems of {w.n_sys}, chi2"
                      f"{' + gradient' if grad else ''}, {el:.2f} s wall"}


def grid_sweep_throughput(kc, synth, dev, stream, args):
    """Mixed chi2 on the 2^20-system sweep (config 2), autotuned."""
    import torch
    w = synth.uniform(2)
    P = torch.tensor(w.params, device=dev)
    T = torch.tensor(w.t, device=dev)
    S = torch.tensor(w.sigma, device=dev)
    V = kc.kc_rv_predict(torch.tensor(w.truth[None, :], device=dev), T)[0]
    V += torch.tensor(w.noise, device=dev)
    out = torch.empty(w.n_sys, dtype=torch.float32, device=dev)
    if not args.no_tune:
        kc.kc_autotune(P, T, V, S, kernel="chi2", mode="mixed", stream=stream)
    for _ in range(2):
        kc.kc_chi2_eval_mixed(P, T, V, S, out=out, stream=stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 5
    hold_gpu(stream, steps * 200.0)
    a.record(stream)
    for _ in range(steps):
        kc.kc_chi2_eval_mixed(P, T, V, S, out=out, stream=stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    sec = a.elapsed_time(b) / 1e3 / steps
    evals = w.n_sys * w.n_pl * w.n_obs
    val = evals / sec
    tile = kc.kc_get_tile("chi2", "mixed", w.n_sys, w.n_pl, w.n_obs)
    fpe = mixed_flops_per_eval(w.n_pl, warp=tile[2] == 3)
    peak = 2 * FP32_LANES_PER_SM * sm_count() * sm_mhz_for_peaks() * 1e6 / 1e12
    out = {"value": val, "unit": "planet-obs evals/s", "ms_per_step": 1e3 * sec,
           "n_sys": w.n_sys, "roofline_frac": val * fpe / 1e12 / peak,
           "roofline": {"bound": "alu", "achieved": val * fpe / 1e12, "peak": peak,
                        "unit": "TFLOP/s", "frac": val * fpe / 1e12 / peak,
                        "flops_per_eval": fpe, "kernel": mixed_kernel_name(w.n_pl, tile)},
           "tile": {"threads_per_system": tile[0], "block": tile[1], "split": tile[2]},
           "inputs": "176 MB of parameters > L2"}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_subset(w, 16384)
    return out


def gradient_throughput(kc, synth, dev, stream, args):
    """Config 3 (65536 systems, n_pl 3, n_obs 512, t0 = 2450000): chi2 and
    its gradient in one adjoint launch, the same plus the Gauss-Newton matrix
    (16 x 16 per system), and the free-jitter log-likelihood with its
    gradient, mixed precision; the FP64 adjoint."""
    import torch
    w = synth.uniform(3)
    P = torch.tensor(w.params, device=dev)
    T = torch.tensor(w.t, device=dev)
    S = torch.tensor(w.sigma, device=dev)
    V = kc.kc_rv_predict(torch.tensor(w.truth[None, :], device=dev), T, t0=w.t0)[0]
    V += torch.tensor(w.noise, device=dev)
    PJ = torch.cat([P, torch.full((w.n_sys, 1), 1.5, dtype=P.dtype, device=dev)], dim=1)
    if not args.no_tune:
        kc.kc_autotune(P, T, V, S, kernel="grad", mode="mixed", stream=stream)
    evals = w.n_sys * w.n_pl * w.n_obs
    out = {"n_sys": w.n_sys, "unit": "planet-obs evals/s"}
    for name, fn in (("chi2_grad", lambda: kc.kc_chi2_grad(P, T, V, S, t0=w.t0, mode="mixed",
                                                           stream=stream)),
                     ("gauss_newton", lambda: kc.kc_chi2_gauss_newton(P, T, V, S, t0=w.t0,
                                                                      mode="mixed",
                                                                      stream=stream)),
                     ("nll_grad", lambda: kc.kc_nll_grad(PJ, T, V, S, t0=w.t0, mode="mixed",
                                                         stream=stream)),
                     ("chi2_grad_fp64", lambda: kc.kc_chi2_grad(P, T, V, S, t0=w.t0,
                                                                mode="fp64", stream=stream)),
                     ) + tuple(
                         (f"gauss_newton_split{split}",
                          lambda split=split: gn_with_split(kc, split, P, T, V, S, w, stream))
                         for split in GN_SPLITS):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2 if name.endswith("fp64") else 5
        hold_gpu(stream, reps * 200.0)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        out[name] = evals * reps / (a.elapsed_time(b) / 1e3)
    peak = 2 * FP32_LANES_PER_SM * sm_count() * sm_mhz_for_peaks() * 1e6 / 1e12
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_subset(w, 16384, grad=True)
    out["roofline_alu"] = {
        "peak": peak, "unit": "TFLOP/s",
        "chi2_grad_frac": out["chi2_grad"] * grad_flops_per_eval(w.n_pl) / 1e12 / peak,
        "nll_grad_frac": out["nll_grad"] * grad_flops_per_eval(w.n_pl) / 1e12 / peak,
        "gauss_newton_frac": out["gauss_newton"] * gn_flops_per_eval(w.n_pl) / 1e12 / peak,
        "flops_per_eval": {"grad": grad_flops_per_eval(w.n_pl), "gauss_newton": gn_flops_per_eval(w.n_pl)},
        "gauss_newton_tensor_tflops": out["gauss_newton"] / w.n_pl * gn_tensor_flops_per_obs(
            w.n_pl, kc.kc_get_tile("gn", "mixed", w.n_sys, w.n_pl, w.n_obs)[2]) / 1e12}
    # the two ways of adding U^T U, side by side
    out["gauss_newton_variants"] = {
        name: out.pop(f"gauss_newton_split{split}")
        for split, name in zip(GN_SPLITS, ("mma_sync", "tcgen05"))}
    out["gauss_newton_default_split"] = kc.kc_get_tile("gn", "mixed", w.n_sys, w.n_pl,
                                                       w.n_obs)[2]
    return out


# Gauss-Newton tile splits: 0 = mma.sync, 4 = tcgen05
GN_SPLITS = (0, 4)


def gn_with_split(kc, split, P, T, V, S, w, stream):
    """One Gauss-Newton launch with the given U^T U variant pinned for the
    workload's size class, the previous table entry restored after."""
    prev = kc.kc_get_tile("gn", "mixed", w.n_sys, w.n_pl, w.n_obs)
    kc.kc_set_tile("gn", "mixed", w.n_sys, w.n_pl, w.n_obs, (32, 128, split))
    try:
        return kc.kc_chi2_gauss_newton(P, T, V, S, t0=w.t0, mode="mixed", stream=stream)
    finally:
        kc.kc_set_tile("gn", "mixed", w.n_sys, w.n_pl, w.n_obs, prev)


def demcmc_throughput(kc, w, P, T, V, S, dev, generations=64):
    """DE-MC (two-half differential evolution) over the batch's 4096 model
    systems as a population: generations per second with graph replay."""
    import torch
    # the library's default chi2 tile for the halves (the autotuner's pick
    # among near-equal tiles moves the rate by a few per cent between runs)
    mc = kc.DEMCMC(P, T, V, S, mode="mixed", eps_scale=1e-6, hop_every=0, seed=5)
    span = 2 * mc.batch                     # generations per graph replay
    mc.run(2 * span)    # eager until the draw buffers align, then one captured span
    generations = max(span, generations // span * span)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_gpu(torch.cuda.current_stream(dev), generations * 300.0)
    a.record()
    mc.run(generations)
    b.record()
    torch.cuda.synchronize(dev)
    sec = a.elapsed_time(b) / 1e3
    return {"generations_per_s": generations / sec, "population": w.n_sys,
            "planet_obs_evals_per_s": generations * w.n_sys * w.n_pl * w.n_obs / sec,
            "acceptance": mc.acceptance}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="kc", choices=["kc", "reference"])
    ap.add_argument("--config", type=int, default=1, choices=[1, 2, 4],
                    help="1: paper-shaped batch (default), 2: 2^20-system sweep, "
                         "4: ragged batch (forward + gradient, one persistent launch)")
    ap.add_argument("--n-sys", type=int, default=None,
                    help="smaller batch of the same distribution (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="use the built-in tile heuristic instead of the autotuner")
    ap.add_argument("--tile", default=None,
                    help="pin threads_per_system,block[,split] for the mixed chi2 kernel")
    ap.add_argument("--no-grad", action="store_true",
                    help="config 4: time the forward plan only")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 / grid-sweep side measurements")
    ap.add_argument("--no-ragged", action="store_true",
                    help="skip the ragged-batch side measurement of the default run")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._thread = None

    def start(self):
        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(
                        ["nvidia-smi", "-i", str(self.index),
                         f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                        capture_output=True, text=True, timeout=5).stdout.strip()
                    if out:
                        self.samples.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._thread = threading.Thread(target=run, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join(timeout=10)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 2 + i and s[2 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ helpers

def dist_setup(args):
    from paper_0812_2976_gb300 import dist as kdist
    return kdist.env()


def peaks():
    try:
        with open(MEASURED) as f:
            return json.load(f), "measured"
    except Exception:
        return {}, "fallback"


def oracle_cpu_baseline(w, seconds=3.0, gpu_chi2=None):
    """Time the FP64 CPU oracle on the host cores over this workload's batch:
    whole batches repeated until ~`seconds` of wall time.  Its observations
    are formed by the oracle itself from the same seeded draws.  With
    gpu_chi2(mode, v_obs) (the library's chi2 of the same batch on those
    observations), also the paper's accuracy figures (Table 2: maximum
    fractional and absolute error, L1 norm of the error) of both paths
    against the oracle over every system of the batch."""
    import oracle
    oracle.build()
    v_obs = oracle.predict(w.truth, w.t, w.n_pl, w.t0)[0] + w.noise
    cores = oracle.max_threads()
    evals_per = w.n_sys * w.n_pl * w.n_obs
    oracle.chi2(w.params[:64], w.t, v_obs, w.sigma, w.n_pl, w.t0)   # warm
    reps, t_start = 0, time.perf_counter()
    while True:
        ref = oracle.chi2(w.params, w.t, v_obs, w.sigma, w.n_pl, w.t0)
        reps += 1
        el = time.perf_counter() - t_start
        if el >= seconds:
            break
    out = {"value": evals_per * reps / el, "unit": "planet-obs evals/s", "cores": cores,
           "kind": "oracle",
           "sample": f"{reps} x the {w.n_sys}-system batch ({evals_per} evals each), "
                     f"{el:.1f} s wall, OpenMP over systems"}
    # one thread as well, the setting of the paper's CPU comparison
    n1 = max(64, w.n_sys // 16)
    oracle.set_threads(1)
    try:
        t1 = time.perf_counter()
        oracle.chi2(w.params[:n1], w.t, v_obs, w.sigma, w.n_pl, w.t0)
        el1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    out["single_thread"] = {"value": n1 * w.n_pl * w.n_obs / el1, "cores": 1,
                            "sample": f"the first {n1} systems, {el1:.2f} s wall"}
    if gpu_chi2 is not None:
        acc = {"systems": int(w.n_sys), "against": "the FP64 CPU oracle on the same inputs"}
        for mode in ("mixed", "fp64"):
            err = np.abs(np.asarray(gpu_chi2(mode, v_obs), dtype=np.float64) - ref)
            acc[mode] = {"max_frac_err": float(np.max(err / np.abs(ref))),
                         "max_abs_err": float(np.max(err)),
                         "l1_rel_err": float(np.sum(err) / np.sum(np.abs(ref)))}
        out["accuracy"] = acc
    return out


# ------------------------------------------------------------------ arms

def run_reference(args):
    """The FP64 CPU oracle as the reference arm, on the host cores."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_0812_2976_gb300 import synth
    oracle.build()
    if args.config == 4:
        return run_reference_ragged(args)
    w = synth.uniform(args.config, n_sys=None if args.config == 1 else 4096)
    v = oracle.predict(w.truth, w.t, w.n_pl, w.t0)[0] + w.noise
    per_step = 256                                  # systems per timed step
    cores = oracle.max_threads()
    for i in range(args.warmup):
        sl = slice((i * per_step) % w.n_sys, (i * per_step) % w.n_sys + per_step)
        oracle.chi2(w.params[sl], w.t, v, w.sigma, w.n_pl, w.t0)
    t0 = time.perf_counter()
    for i in range(args.steps):
        s0 = (i * per_step) % w.n_sys
        oracle.chi2(w.params[s0:s0 + per_step], w.t, v, w.sigma, w.n_pl, w.t0)
    el = time.perf_counter() - t0
    evals = args.steps * per_step * w.n_pl * w.n_obs
    value = evals / el
    line = {
        "impl": "reference", "metric": METRIC_PAPER_BATCH,
        "value": value, "unit": "planet-obs evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.shape.name, "n_sys_per_step": per_step, "n_pl": w.n_pl,
                   "n_obs": w.n_obs},
        "cpu_baseline": {"value": value, "unit": "planet-obs evals/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{per_step} systems of the {w.shape.name} batch per step"},
        "e2e": {"value": value, "unit": "planet-obs evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_ragged(args):
    """The oracle on the ragged workload: each step a 200-system sample."""
    import oracle
    from paper_0812_2976_gb300 import synth
    w = synth.ragged()
    cores = oracle.max_threads()
    per_step = 200
    rng = np.random.default_rng(0)
    subs = []
    for _ in range(args.warmup + args.steps):
        sub = synth.subset_ragged(w, np.sort(rng.choice(w.n_sys, per_step, replace=False)))
        v = oracle.predict_ragged(sub.truth, sub.par_off, sub.n_pl, sub.t, sub.obs_off) + sub.noise
        subs.append((sub, v))
    for sub, v in subs[:args.warmup]:
        oracle.chi2_ragged(sub.params, sub.par_off, sub.n_pl, sub.t, v, sub.sigma, sub.obs_off,
                           grad=True)
    evals, t0 = 0, time.perf_counter()
    for sub, v in subs[args.warmup:]:
        oracle.chi2_ragged(sub.params, sub.par_off, sub.n_pl, sub.t, v, sub.sigma, sub.obs_off,
                           grad=True)
        evals += sub.evals()
    el = time.perf_counter() - t0
    value = evals / el
    print(json.dumps({
        "impl": "reference",
        "metric": "planet-obs evals/s (chi2 + gradient, ragged n_pl 1-6, n_obs 16-1024)",
        "value": value, "unit": "planet-obs evals/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ragged", "n_sys_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "planet-obs evals/s", "cores": cores,
                         "kind": "oracle", "sample": f"{per_step} random systems per step"},
        "e2e": {"value": value, "unit": "planet-obs evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_kc(args):
    import torch
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    import paper_0812_2976_gb300 as kc
    from paper_0812_2976_gb300 import build, synth
    build.build()
    kc._lib.load()

    # each rank its own batch of the same shape (a shard of a larger sweep)
    w = synth.uniform(args.config, n_sys=args.n_sys,
                      seed=synth.SEED_BASE + args.config + 1000 * rank if rank else None)
    P = torch.tensor(w.params, device=dev)
    T = torch.tensor(w.t, device=dev)
    S = torch.tensor(w.sigma, device=dev)
    truth = torch.tensor(w.truth[None, :], device=dev)
    V = kc.kc_rv_predict(truth, T, t0=w.t0)[0] + torch.tensor(w.noise, device=dev)
    out = torch.empty(w.n_sys, dtype=torch.float32, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream(dev)
    evals = w.n_sys * w.n_pl * w.n_obs

    tile_kind = "heuristic"
    if args.tile:
        kc.kc_set_tile("chi2", "mixed", w.n_sys, w.n_pl, w.n_obs,
                       tuple(int(x) for x in args.tile.split(",")))
        tile_kind = "pinned"
    tile = kc.kc_get_tile("chi2", "mixed", w.n_sys, w.n_pl, w.n_obs)
    if not args.no_tune and not args.tile:
        tile, _ = kc.kc_autotune(P, T, V, S, kernel="chi2", mode="mixed", stream=stream)
        tile_kind = "autotuned"

    # a pool of copies of the step's inputs, together larger than L2: step i
    # reads copy i mod n_sets, untouched for n_sets - 1 steps and 256 MiB
    set_bytes = sum(x.numel() * x.element_size() for x in (P, T, V, S))
    n_sets = max(2, -(-ROTATE_BYTES // set_bytes))
    pool = [(P, T, V, S)] + [tuple(x.clone() for x in (P, T, V, S))
                             for _ in range(n_sets - 1)]

    def step(i=0):
        p, t, v, s = pool[i % n_sets]
        kc.kc_chi2_eval_mixed(p, t, v, s, out=out, stream=stream)

    for i in range(max(args.warmup, 3)):
        step(n_sets - 1 - i)
    flush.fill_(0)
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local) if rank == 0 else None
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
    # K steps back to back (the timed region)
    hold_gpu(stream, args.steps * 200.0)
    t0e.record(stream)
    for i in range(args.steps):
        step(i)
    t1e.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    # the same K steps, each between its own events after an L2 flush
    hold_gpu(stream, args.steps * 300.0)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                      # cold L2 for every step
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    t_sum = t0e.elapsed_time(t1e) / 1e3
    t_flushed = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    if world > 1:
        from paper_0812_2976_gb300 import dist as kdist
        t_sum = kdist.max_over_ranks(t_sum, device=dev)
        t_flushed = kdist.max_over_ranks(t_flushed, device=dev)
    value = evals * args.steps * world / t_sum
    ms_per_step = 1e3 * t_sum / args.steps
    per_step_flushed = {
        "value": evals * args.steps * world / t_flushed, "unit": "planet-obs evals/s",
        "ms_per_step": 1e3 * t_flushed / args.steps,
        "how": "the same steps, each between its own CUDA events with L2 flushed before it "
               "(write 256 MiB, then read 256 MiB)"}

    # end-to-end through the public API from pinned host memory: the step's
    # inputs (parameters, times, velocities, uncertainties) packed in one
    # pinned buffer and sent with one copy into one device buffer, whose
    # views the library reads; chi2 comes back with one copy.  Steps
    # alternate between two streams and two sets of device and pinned
    # output buffers, as a serving loop would drive the library: one step's
    # copies overlap the other's kernel, while each kernel waits for the
    # previous step's (kernels never overlap one another).  Timed from the
    # first copy of the first step to the last read of the last (CUDA
    # events, both streams joined), every step's copies inside; no L2 flush
    # between the steps (each step's inputs arrive fresh from the host)
    n_par, n_obs = P.numel(), T.numel()
    hbuf = torch.cat([torch.tensor(w.params).ravel(), T.cpu(), V.cpu(), S.cpu()]).pin_memory()
    pipe = [stream, torch.cuda.Stream(dev)]
    bufs = []
    for _ in pipe:
        dbuf = torch.empty_like(hbuf, device=dev)
        views = (dbuf[:n_par].view(P.shape),) + tuple(
            dbuf[n_par + i * n_obs:n_par + (i + 1) * n_obs] for i in range(3))
        bufs.append((dbuf, views, torch.empty(w.n_sys, dtype=torch.float32, device=dev),
                     torch.empty(w.n_sys, dtype=torch.float32).pin_memory()))

    kernel_done = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_step(i):
        st = pipe[i % 2]
        dbuf, (dP, dT, dV, dS), dout, hout = bufs[i % 2]
        with torch.cuda.stream(st):
            dbuf.copy_(hbuf, non_blocking=True)
            if i > 0:
                st.wait_event(kernel_done[(i - 1) % 2])      # the previous step's kernel
            kc.kc_chi2_eval_mixed(dP, dT, dV, dS, out=dout, stream=st)
            kernel_done[i % 2].record(st)
            hout.copy_(dout, non_blocking=True)

    def e2e_run(n):
        """n pipelined steps between two events on the first stream."""
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        joined = torch.cuda.Event()
        t0e.record(pipe[0])
        pipe[1].wait_event(t0e)
        for i in range(n):
            e2e_step(i)
        joined.record(pipe[1])
        pipe[0].wait_event(joined)
        t1e.record(pipe[0])
        return t0e, t1e

    e2e_run(4)
    torch.cuda.synchronize(dev)
    hold_gpu(stream, args.steps * 400.0)
    t0e, t1e = e2e_run(args.steps)
    torch.cuda.synchronize(dev)
    e2e_s = t0e.elapsed_time(t1e) / 1e3
    if world > 1:
        from paper_0812_2976_gb300 import dist as kdist
        e2e_s = kdist.max_over_ranks(e2e_s, device=dev)
    h2d = hbuf.numel() * 8
    d2h = w.n_sys * 4
    e2e = {"value": evals * args.steps * world / e2e_s, "unit": "planet-obs evals/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "how": "steps alternating between two streams (copies of one overlap the other's "
                  "kernel; each kernel after the previous one), CUDA events from the first "
                  "copy to the last read, no L2 flush (each step's inputs reach its kernel "
                  "through L2 from its own copy)"}

    # the same steps fully serialised on one stream, each between its own
    # CUDA events with L2 flushed before it (the device-resident value's
    # timing with the copies added)
    def serial_step():
        dbuf0, (dP0, dT0, dV0, dS0), dout0, hout0 = bufs[0]
        dbuf0.copy_(hbuf, non_blocking=True)
        kc.kc_chi2_eval_mixed(dP0, dT0, dV0, dS0, out=dout0, stream=stream)
        hout0.copy_(dout0, non_blocking=True)

    serial_s = time_steps(serial_step, args.steps, stream, flush)
    if world > 1:
        from paper_0812_2976_gb300 import dist as kdist
        serial_s = kdist.max_over_ranks(serial_s, device=dev)
    e2e["serialised"] = {"value": evals * args.steps * world / serial_s,
                         "ms_per_step": 1e3 * serial_s / args.steps,
                         "how": "each step's copy in, kernel and copy out on one stream between "
                                "its own CUDA events, L2 flushed before every step"}

    # the same steps on the host's clock: back-to-back calls through the
    # binding and the C ABI (ctypes, argument checks, launch) with their
    # copies on one stream, one synchronise at the end; no GPU hold, no L2
    # flush (the host's cost per call is what this measures)
    dbuf0, (dP0, dT0, dV0, dS0), dout0, hout0 = bufs[0]

    def wall_step():
        dbuf0.copy_(hbuf, non_blocking=True)
        kc.kc_chi2_eval_mixed(dP0, dT0, dV0, dS0, out=dout0, stream=stream)
        hout0.copy_(dout0, non_blocking=True)

    for _ in range(3):
        wall_step()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        wall_step()
    torch.cuda.synchronize(dev)
    wall_s = time.perf_counter() - wall0
    if world > 1:
        from paper_0812_2976_gb300 import dist as kdist
        wall_s = kdist.max_over_ranks(wall_s, device=dev)
    e2e_wall = {"value": evals * args.steps * world / wall_s, "unit": "planet-obs evals/s",
                "ms_per_step": 1e3 * wall_s / args.steps,
                "how": "time.perf_counter around the steps of the e2e leg issued back to back "
                       "on one stream (H2D copy, kc_chi2_eval_mixed, D2H copy), final "
                       "synchronise included"}

    extras = {}
    if not args.no_extras:
        # FP64 path on the same batch ("mixed vs FP64")
        out64 = torch.empty(w.n_sys, dtype=torch.float64, device=dev)
        if not args.no_tune:
            kc.kc_autotune(P, T, V, S, kernel="chi2", mode="fp64", stream=stream)
        for _ in range(3):
            kc.kc_chi2_eval(P, T, V, S, out=out64, stream=stream)
        f_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(min(args.steps, 20))]
        hold_gpu(stream, len(f_ev) * 300.0)
        for a, b in f_ev:
            flush.fill_(1)
            a.record(stream)
            kc.kc_chi2_eval(P, T, V, S, out=out64, stream=stream)
            b.record(stream)
        torch.cuda.synchronize(dev)
        f_s = sum(a.elapsed_time(b) for a, b in f_ev) / 1e3
        f64_val = evals * len(f_ev) / f_s
        # FP64 peak: DFMA rate per SM per clock measured live by the library's
        # pipe probe, x 2 FLOP x SMs x maximum SM clock
        f64_rate = kc.kc_measure_pipe_rate("fp64", stream=stream)
        f32_rate = kc.kc_measure_pipe_rate("fp32", stream=stream)
        f64_peak = 2 * f64_rate * sm_count() * sm_mhz_for_peaks() * 1e6 / 1e12
        extras["fp64"] = {"value": f64_val, "unit": "planet-obs evals/s",
                          "ms_per_step": 1e3 * f_s / len(f_ev),
                          "roofline": {"bound": "fp64", "achieved": f64_val * F64_FLOPS_PER_EVAL
                                       / 1e12, "peak": f64_peak, "unit": "TFLOP/s",
                                       "frac": f64_val * F64_FLOPS_PER_EVAL / 1e12 / f64_peak,
                                       "flops_per_eval": F64_FLOPS_PER_EVAL,
                                       "peak_basis": f"measured DFMA rate {f64_rate:.2f} per SM "
                                                     f"per clock x 2 FLOP x {sm_count()} SMs x max SM clock"}}
        extras["pipe_rates_per_sm_clock"] = {"fp32_fma": f32_rate, "fp64_fma": f64_rate}
        extras["kepler_only"] = kepler_throughput(kc, dev, stream)
        extras["grid_sweep"] = grid_sweep_throughput(kc, synth, dev, stream, args)
        extras["gradient"] = gradient_throughput(kc, synth, dev, stream, args)
        extras["demcmc"] = demcmc_throughput(kc, w, P, T, V, S, dev)
        if world == 1 and not args.no_ragged:
            extras["ragged"] = ragged_measure(kc, synth, dev, stream, flush, args, compact=True)

    pk, pk_kind = peaks()
    sm_mhz = pk.get("sm_max_mhz", FALLBACK_SM_MHZ)
    peak_tflops = 2 * FP32_LANES_PER_SM * sm_count() * sm_mhz * 1e6 / 1e12
    warp = tile[2] == 3
    flops = mixed_flops_per_eval(w.n_pl, warp) * evals
    achieved = flops / (t_sum / args.steps) / 1e12          # one GPU's launch
    traffic = (DRAM_BYTES_PER_LAUNCH.get((args.config, args.n_sys, tuple(tile)))
               if world == 1 else None)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                "kernel": mixed_kernel_name(w.n_pl, tile),
                "peak_basis": f"FP32 FMA pipe: {sm_count()} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP "
                              f"x {sm_mhz:.0f} MHz ({pk_kind} max SM clock)",
                "flops_per_eval": mixed_flops_per_eval(w.n_pl, warp)}

    if rank != 0:
        return
    line = {
        "metric": METRIC_PAPER_BATCH,
        "value": value, "unit": "planet-obs evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ds (mixed)",
        "data": "synthetic",
        "config": {"workload": w.shape.name, "n_sys": w.n_sys, "n_pl": w.n_pl,
                   "n_obs": w.n_obs, "per_rank": True,
                   "l2": f"inputs larger than L2: each step its own copy of the inputs from a "
                         f"pool of {n_sets} ({n_sets * set_bytes / 2**20:.0f} MiB), steps back to "
                         f"back between one pair of CUDA events, no flush",
                   "tile": {"threads_per_system": tile[0], "block": tile[1],
                            "split": tile[2], "how": tile_kind}},
        "roofline": roofline,
        "per_step_flushed": per_step_flushed,
        "e2e": e2e,
        "e2e_wall": e2e_wall,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    line.update(extras)
    if not args.no_cpu_baseline and world == 1:
        def gpu_chi2(mode, v_obs):
            vo = torch.tensor(v_obs, device=dev)
            if mode == "mixed":
                return kc.kc_chi2_eval_mixed(P, T, vo, S).cpu().numpy()
            return kc.kc_chi2_eval(P, T, vo, S).cpu().numpy()
        line["cpu_baseline"] = oracle_cpu_baseline(w, gpu_chi2=gpu_chi2)
        line["accuracy"] = line["cpu_baseline"].pop("accuracy")
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


class L2Flush:
    """Evicts L2 between timed steps: write one buffer larger than L2, then
    read another, so no dirty line is left for the next kernel to write
    back."""

    def __init__(self, dev, nbytes=256 << 20):
        import torch
        self.a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.b = torch.ones(nbytes // 4, dtype=torch.float32, device=dev)
        # first use loads the fill and reduction kernels (a host stall of up
        # to a second): done here, outside every timed loop
        for v in range(2):
            self.fill_(v)
        torch.cuda.synchronize(dev)

    def fill_(self, v):
        self.a.fill_(v)
        self.b.sum()


def time_steps(fn, steps, stream, flush):
    """Sum of per-step CUDA-event times of fn() with a cold L2 each step."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    hold_gpu(stream, steps * 400.0)
    for i, (a, b) in enumerate(ev):
        flush.fill_(i & 0xFF)
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / 1e3


def run_kc_ragged(args):
    """Config 4 as the headline: 200000 systems with their own n_obs ~
    U[16,1024] and n_pl ~ U{1..6}; one step = forward chi2 + gradient of
    every system in one persistent, graph-replayed launch (kc_plan_run)."""
    import torch
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_0812_2976_gb300 as kc
    from paper_0812_2976_gb300 import build, synth
    build.build()
    kc._lib.load()
    stream = torch.cuda.current_stream(dev)
    flush = L2Flush(dev)
    r = ragged_measure(kc, synth, dev, stream, flush, args, world=world, rank=rank)
    if rank != 0:
        return
    want_grad = not args.no_grad
    line = {
        "metric": ("planet-obs evals/s (chi2 + gradient, ragged n_pl 1-6, n_obs 16-1024)"
                   if want_grad else "planet-obs evals/s (chi2, ragged n_pl 1-6, n_obs 16-1024)"),
        "value": r["value"], "unit": "planet-obs evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+ds (mixed)", "data": "synthetic", "config": r["config"],
        "e2e": r["e2e"], "gpu_launches": args.steps, "clocks": r["clocks"],
        "roofline": r["roofline"]}
    for k in ("forward_only", "padded_baseline", "cpu_baseline"):
        if k in r:
            line[k] = r[k]
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def ragged_measure(kc, synth, dev, stream, flush, args, world=1, rank=0, compact=False):
    """The ragged workload (config 4) through a RaggedPlan: chi2 + gradient
    of every system per step (chi2 only with --no-grad), with the forward-
    only plan, the padded uniform-size baseline, the ALU roofline of the
    persistent kernel, end to end from pinned host memory and the oracle on
    a sample of at least 16384 systems.  compact: the dictionary kept as an
    extra of the default run."""
    import torch
    w = synth.ragged(n_sys=args.n_sys if args.config == 4 and args.n_sys else synth.RAGGED_N_SYS,
                     seed=None if rank == 0 else synth.SEED_BASE + 4 + 1000 * rank)
    T = torch.tensor(w.t, device=dev)
    S = torch.tensor(w.sigma, device=dev)
    V = kc.kc_rv_predict_ragged(torch.tensor(w.truth, device=dev), torch.tensor(w.par_off),
                                torch.tensor(w.n_pl), T, torch.tensor(w.obs_off))
    V += torch.tensor(w.noise, device=dev)
    P = torch.tensor(w.params, device=dev)
    evals = w.evals()
    want_grad = not args.no_grad

    plan = kc.RaggedPlan(w.obs_off, w.n_pl, mode="mixed", want_grad=want_grad)
    plan.set_observations(T, V, S)
    shape = plan.autotune(P) if not args.no_tune else None
    res = plan.run(P)
    chi, grad = res if want_grad else (res, None)
    for _ in range(max(args.warmup, 3)):
        plan.run(P, chi, grad)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index) if rank == 0 and not compact else None
    if world > 1:
        torch.distributed.barrier()
    if sampler:
        sampler.start()
    t_sum = time_steps(lambda: plan.run(P, chi, grad), args.steps, stream, flush)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    if world > 1:
        from paper_0812_2976_gb300 import dist as kdist
        t_sum = kdist.max_over_ranks(t_sum, device=dev)
    out = {"value": evals * args.steps * world / t_sum, "unit": "planet-obs evals/s",
           "ms_per_step": 1e3 * t_sum / args.steps, "clocks": clocks,
           "what": "chi2 + gradient" if want_grad else "chi2",
           "config": {"workload": "ragged", "n_sys": w.n_sys, "evals": evals,
                      "n_obs_total": int(w.obs_off[-1]),
                      "l2": "flushed between steps (write 256 MiB, then read 256 MiB)",
                      "launch": {"block": shape[0], "ctas_per_sm": shape[1], "how": "autotuned"}
                      if shape else "default"}}
    # ALU roofline of the persistent kernel: every system at its own n_pl
    n_obs_s = np.diff(np.asarray(w.obs_off)).astype(np.float64)
    npl_s = np.asarray(w.n_pl).astype(np.float64)
    per_planet = (grad_flops_per_eval(1) - 12.0) if want_grad else (mixed_flops_per_eval(1) - 10.0)
    per_obs = 12.0 if want_grad else 10.0
    flops_step = float(np.sum(n_obs_s * (npl_s * per_planet + per_obs)))
    peak = 2 * FP32_LANES_PER_SM * sm_count() * sm_mhz_for_peaks() * 1e6 / 1e12
    achieved = flops_step / (t_sum / args.steps) / 1e12
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak, "traffic": None,
                       "kernel": f"ragged_mixed_kernel<{'GRAD' if want_grad else 'FWD'}>",
                       "flops_per_step": flops_step}

    # end to end: host parameters in, host chi2 + gradient out (the plan
    # writes both into views of one device buffer, returned with one copy);
    # steps alternate between two streams (the plan keeps a work queue and a
    # graph per stream) so that one step's copies overlap the other's
    # kernel, each kernel after the previous one; CUDA events from the first
    # copy to the last read
    hP = torch.tensor(w.params).pin_memory()
    n_out = chi.numel() + (grad.numel() if want_grad else 0)
    pipe = [stream, torch.cuda.Stream(dev)]
    bufs = []
    for _ in pipe:
        dP = torch.empty_like(P)
        dout = torch.empty(n_out, dtype=chi.dtype, device=dev)
        bufs.append((dP, dout, dout[:chi.numel()], dout[chi.numel():] if want_grad else None,
                     torch.empty(n_out, dtype=chi.dtype).pin_memory()))

    kernel_done = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_step(i):
        st = pipe[i % 2]
        dP, dout, echi, egrad, hout = bufs[i % 2]
        with torch.cuda.stream(st):
            dP.copy_(hP, non_blocking=True)
            if i > 0:
                st.wait_event(kernel_done[(i - 1) % 2])      # the previous step's kernel
            plan.run(dP, echi, egrad, stream=st)
            kernel_done[i % 2].record(st)
            hout.copy_(dout, non_blocking=True)

    def e2e_run(n):
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        joined = torch.cuda.Event()
        t0e.record(pipe[0])
        pipe[1].wait_event(t0e)
        for i in range(n):
            e2e_step(i)
        joined.record(pipe[1])
        pipe[0].wait_event(joined)
        t1e.record(pipe[0])
        return t0e, t1e

    e2e_run(4)                                  # captures each stream's graph
    torch.cuda.synchronize(dev)
    hold_gpu(stream, args.steps * 400.0)
    t0e, t1e = e2e_run(args.steps)
    torch.cuda.synchronize(dev)
    e2e_s = t0e.elapsed_time(t1e) / 1e3
    out["e2e"] = {"value": evals * args.steps / e2e_s, "unit": "planet-obs evals/s",
                  "h2d_bytes_per_step": hP.numel() * 8,
                  "d2h_bytes_per_step": n_out * chi.element_size(),
                  "how": "steps alternating between two streams, each kernel after the "
                         "previous one, CUDA events from the first copy to the last read"}
    del plan, bufs, hP, chi, grad

    if not args.no_extras or compact:
        out.update(ragged_extras(args, kc, synth, w, P, T, V, S, evals, stream, flush, dev))
    if not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        idx = np.arange(0, w.n_sys, max(1, w.n_sys // 16384))     # >= 16384 systems
        sub = synth.subset_ragged(w, idx)
        vsub = oracle.predict_ragged(sub.truth, sub.par_off, sub.n_pl, sub.t,
                                     sub.obs_off) + sub.noise
        t0c = time.perf_counter()
        oracle.chi2_ragged(sub.params, sub.par_off, sub.n_pl, sub.t, vsub, sub.sigma,
                           sub.obs_off, grad=want_grad)
        el = time.perf_counter() - t0c
        out["cpu_baseline"] = {"value": sub.evals() / el, "unit": "planet-obs evals/s",
                               "cores": oracle.max_threads(), "kind": "oracle",
                               "sample": f"{idx.size} systems (every {idx[1] - idx[0]}th), "
                                         f"chi2{' + gradient' if want_grad else ''}, "
                                         f"{el:.1f} s wall"}
    del P, T, V, S
    torch.cuda.empty_cache()
    if compact:
        out.pop("clocks", None)
    return out


def ragged_extras(args, kc, synth, w, P, T, V, S, evals, stream, flush, dev):
    """Forward-only plan, and the padded uniform-size baseline: the same
    kernel with every system padded to n_pl = 6 (K = 0) and n_obs = 1024
    (zero weight), throughput counted in useful evaluations."""
    import torch
    out = {}
    fplan = kc.RaggedPlan(w.obs_off, w.n_pl, mode="mixed")
    fplan.set_observations(T, V, S)
    if not args.no_tune:
        fplan.autotune(P)
    fchi = fplan.run(P)
    fwd_s = time_steps(lambda: fplan.run(P, fchi), args.steps, stream, flush)
    out["forward_only"] = {"value": evals / (fwd_s / args.steps), "unit": "planet-obs evals/s"}
    del fplan
    pw, pv = synth.pad_ragged(w, V.cpu().numpy(), n_pl=6, n_obs=1024)
    pplan = kc.RaggedPlan(pw.obs_off, pw.n_pl, mode="mixed", want_grad=not args.no_grad)
    pT, pV, pS = (torch.tensor(pw.t, device=dev), torch.tensor(pv, device=dev),
                  torch.tensor(pw.sigma, device=dev))
    pplan.set_observations(pT, pV, pS)
    PP = torch.tensor(pw.params, device=dev)
    if not args.no_tune:
        pplan.autotune(PP)
    res = pplan.run(PP)
    pchi, pgrad = res if not args.no_grad else (res, None)
    pad_steps = max(3, args.steps // 4)
    pad_s = time_steps(lambda: pplan.run(PP, pchi, pgrad), pad_steps, stream, flush)
    out["padded_baseline"] = {"value": evals / (pad_s / pad_steps),
                              "unit": "planet-obs evals/s (useful)",
                              "padded_evals": int(pw.n_sys * 6 * 1024),
                              "ms_per_step": 1e3 * pad_s / pad_steps}
    del pplan
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == 4:
        run_kc_ragged(args)
    else:
        run_kc(args)


if __name__ == "__main__":
    main()
