"""Benchmark of the coupled LBM + WENO5 step (GLUPS and fraction of the HBM roofline).

Default workload: 2D D2Q9, 2048 x 4096 lattice, FP32 populations stored as
f - w_i, FP32 WENO5, A = 1e-5, Vs = 1e-3, kappa = 1e-3, tau = 0.6; synthetic tanh
interface at 0.75 H with a seeded U(-1e-3, 1e-3) perturbation.  One "step" is one
full coupled time step over the whole lattice.  GLUPS = nodes x steps / s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one rank per GPU): independent replicas, one per GPU, no
collective on the data path; the value is the sum over ranks (weak scaling).
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
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

from paper_2106_07694_gb300 import workloads  # noqa: E402

WORKLOADS = {
    "2d": (workloads.MAIN_2D, "coupled LBM+WENO5 GLUPS (2D D2Q9 2048x4096 FP32)", "D2Q9"),
    "3d": (workloads.MAIN_3D, "coupled LBM+WENO5 GLUPS (3D D3Q19 256x256x512 FP32)", "D3Q19"),
    "sugar": (workloads.SUGAR_2D, "coupled LBM+WENO5+sugar GLUPS (2D D2Q9 2048x4096 FP32, two-layer state)",
              "D2Q9"),
    "small": (workloads.SMALL_2D, "coupled LBM+WENO5 GLUPS (2D D2Q9 128x256 FP64, L2-resident parity case)",
              "D2Q9"),
    "weno3": (workloads.WENO3_2D, "coupled LBM+WENO3 GLUPS (2D D2Q9 2048x4096 FP32, paper-literal WENO3)", "D2Q9"),
    "signsplit": (workloads.SIGN_SPLIT_2D,
                  "coupled LBM+WENO5 GLUPS (2D D2Q9 2048x4096 FP32, sign-upwind stencil choice)", "D2Q9"),
    "classes": (workloads.CLASSES_2D,
                "coupled LBM+WENO5 GLUPS (2D D2Q9 2048x4096 FP32, three particle classes)", "D2Q9"),
}
WL, METRIC, LATTICE = WORKLOADS["2d"]
ADJOINT_METRIC = ("gradient of the deposited mass wrt c0 and Vs, GLUPS of the reverse-mode pass "
                  "(2D D2Q9 512x1024 FP32, 2000 steps, checkpoint every 100)")
# launch form of the batched sweep (lbm_wenoc_batch_set_persistent): 1 all phases in one
# persistent launch per 16 steps, 2 grouped fluid launch + persistent stage launch per step
BATCH_MODE = 1
BATCH_FORMS = {0: "grouped", 1: "persistent", 2: "split"}
BATCH_METRIC = "coupled LBM+WENO5 GLUPS, batched sweep of 64 D2Q9 FP32 instances (256x512..1024x2048)"
UNIT = "GLUPS"


# flops per node of one adj_faces launch, counted on the formulation: per WENO5 value and
# its five partial derivatives 131 (candidates 15, differences 21, indicators 15 + 3
# reciprocals, weights 12, value 5, sensitivity factors 18, derivatives 42), per face two
# of them + split values 30 + derivative assembly 74 = 366, two faces per node + scaled
# velocities and face adjoints 34
ADJ_FACES_FLOP = 766


def sm_count(dev=None):
    """Streaming multiprocessors of the device (152 on a GB300)."""
    try:
        import torch
        return int(torch.cuda.get_device_properties(dev if dev is not None else 0).multi_processor_count)
    except Exception:
        return 152


def fp32_peak_tflops(clk, sms=None):
    """FP32 ALU peak derived from the unit counts: SMs x 128 lanes x 2 flop x SM clock."""
    sm_hz = ((clk or {}).get("sm_mhz") or 2070.0) * 1e6
    return (sms or sm_count()) * 128 * 2 * sm_hz / 1e12


def phys_kwargs(wl):
    kw = dict(tau=wl.tau, gravity=wl.gravity, density_contrast=wl.density_contrast,
              settling_velocity=wl.settling_velocity, diffusivity=wl.diffusivity, **wl.sugar, **wl.scheme)
    if wl.class_vs:
        kw["class_vs"] = wl.class_vs
    return kw


def set_classes(sim, wl, to=lambda a: a):
    """Class fields of a polydisperse workload (after init, which puts c0 in class 0)."""
    for k, ck in enumerate(wl.initial_classes() if wl.class_vs else []):
        sim.set_class(k, to(ck))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons: one reading right before the timed region,
    samples every 200 ms during it, one reading right after it (a short region still gets
    two readings)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def _once(self):
        try:
            out = subprocess.run(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                  "-i", str(self.dev)], capture_output=True, text=True, timeout=10).stdout
            self.lines.extend(ln.strip() for ln in out.splitlines() if ln.strip())
        except Exception:
            pass

    def start(self):
        self._once()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
        self._once()
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the ncu
# launch lists summarised in profiles/ (the bench command itself, one pass per launch), with
# the SHA-1 prefix of the kernel sources they were taken on (the kernel's file and the
# headers it includes, concatenated in this order); a changed kernel reports null until it
# is captured again.  The fluid entry is the mean of the two AA parities.
_CSRC = "paper_2106_07694_gb300/csrc/"
_LBM_SRC = ("lbm_kernels.cuh", "lattice.cuh", "common.cuh")
_STAGE_SRC = ("transport_stage2d_wide.cuh", "transport_stage2d.cuh", "transport_sweep2d.cuh", "reduce_kernels.cuh",
              "common.cuh")
_STAGE3D_SRC = ("transport_sweep3d_wide.cuh", "transport_sweep3d.cuh") + _STAGE_SRC
NCU_TRAFFIC = {
    "lbm_collide_stream": (643.1e6, _LBM_SRC, "2097009c2aa4"),
    "rk_stage1": (134.3e6, _STAGE_SRC, "dd1ee704fac2"),
    "rk_stage2": (178.4e6, _STAGE_SRC, "dd1ee704fac2"),
    "rk_stage3": (171.9e6, _STAGE_SRC, "dd1ee704fac2"),
    # 512 x 1024 adjoint workload (the face records stay in L2)
    "adj_faces": (8.57e6, ("adjoint.cuh",) + _LBM_SRC, "d60661f5666e"),
}
# the 256 x 256 x 512 D3Q19 workload
NCU_TRAFFIC_3D = {
    "lbm_collide_stream": (5577.75e6, _LBM_SRC, "2097009c2aa4"),
    "rk_stage1": (966.4e6, _STAGE3D_SRC, "5a04479acddc"),
    "rk_stage2": (1127.2e6, _STAGE3D_SRC, "5a04479acddc"),
    "rk_stage3": (1109.2e6, _STAGE3D_SRC, "5a04479acddc"),
}


def source_hash(files):
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, _CSRC + f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def kernel_traffic(name, table=None):
    table = NCU_TRAFFIC if table is None else table
    if name not in table:
        return None
    nbytes, files, sha = table[name]
    try:
        cur = source_hash(files)
    except OSError:
        return None
    return nbytes if cur == sha else None


def run_oracle_sample(wl, steps, threads):
    """Time the FP64 CPU oracle for `steps` steps (after 1 warm-up): the full 2D lattice,
    or a 64-node-high slab of the 3D one (the full 3D oracle state would need 12 GB)."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle
    if len(wl.shape) == 3:
        wl = wl.with_(shape=(wl.shape[0], wl.shape[1], 64))
    s = oracle.OracleSim(wl.shape, **phys_kwargs(wl))
    s.init(wl.initial_c())
    if wl.sugar:
        s.set_sugar(wl.initial_S())
    set_classes(s, wl)
    s.step(1)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return wl.nodes * steps / dt / 1e9, dt


def bench_reference(args):
    """The oracle as it stands, on the host cores.  Each step is one full coupled step
    of a bounded sample of the workload: the full 2048-wide lattice cut to 128 rows
    (same physics, interface at 0.75 of the band), so K steps end within minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    os.environ["OMP_NUM_THREADS"] = str(threads)
    import oracle
    # a band of the full horizontal extent, 128 nodes high (2D) / 32 high (3D)
    band = WL.with_(shape=tuple(WL.shape[:-1]) + ((128 if len(WL.shape) == 2 else 32),))
    s = oracle.OracleSim(band.shape, **phys_kwargs(band))
    s.init(band.initial_c())
    if band.sugar:
        s.set_sugar(band.initial_S())
    set_classes(s, band)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    total = time.perf_counter() - t0
    value = band.nodes * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WL.name, "shape": list(WL.shape), "lattice": LATTICE,
                                        "host_threads": threads, "sample_shape": list(band.shape)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"FP64 C oracle, {'x'.join(map(str, band.shape))} band of the "
                                   f"workload, {args.steps} steps after {args.warmup} warm-up"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2106_07694_gb300 import build as lbuild
    lbuild.build()
    from paper_2106_07694_gb300 import lbm_wenoc as lw

    def barrier():
        if world > 1:
            dist.barrier()

    wl = WL
    kw = phys_kwargs(wl)
    stream = torch.cuda.current_stream()
    fp64 = wl.dtype == "f64"
    np_dt = np.float64 if fp64 else np.float32
    sim = lw.Simulation(wl.shape, fp64=fp64, stream=stream, **kw)
    c0 = wl.initial_c().astype(np_dt)
    S0 = wl.initial_S().astype(np_dt) if wl.sugar else None
    sim.init(torch.from_numpy(c0).to(dev))
    if S0 is not None:
        sim.set_sugar(torch.from_numpy(S0).to(dev))
    set_classes(sim, wl, lambda a: torch.from_numpy(a.astype(np_dt)).to(dev))
    sim.step(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K coupled steps, production path (CUDA graphs), inputs resident
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = lw.lbm_wenoc_launch_count(sim.handle)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = lw.lbm_wenoc_launch_count(sim.handle) - launches0
    st = sim.status()
    if st != lw.LW_OK:
        raise RuntimeError(f"device status {st} after the timed region")
    from paper_2106_07694_gb300.replicas import job_time_ms, replica_glups
    value, t_max = replica_glups(ms, wl.nodes, args.steps, device=dev)

    # ---- per-kernel durations: the same K steps again, CUDA events around each launch
    lw.lbm_wenoc_profile_enable(sim.handle, True)
    lw.lbm_wenoc_profile_read(sim.handle, reset=True)
    sim.step(args.steps)
    stats = lw.lbm_wenoc_profile_read(sim.handle, reset=True)
    lw.lbm_wenoc_profile_enable(sim.handle, False)
    kernels = {k: {"launches": n, "avg_us": 1e3 * t / max(n, 1), "share": None} for k, (n, t) in stats.items()}
    tot = sum(t for (_, t) in stats.values())
    for k, (n, t) in stats.items():
        kernels[k]["share"] = t / tot if tot > 0 else None
    dominant = max(stats.items(), key=lambda kv: kv[1][1])[0] if stats else None
    peak, peak_kind = load_peaks()
    step_ms = t_max / args.steps
    # Algorithmic work per node (FP32), counted on the textbook formulation:
    #   fluid kernel   2 Q 4 B populations in and out + 4 B c in (D2Q9 76 B, D3Q19 156 B)
    #   RK3 transport  3 stages x dim faces x (2 WENO5-JS reconstructions of 70 flop + split
    #                  fluxes, diffusion, sum) + divergence and Shu-Osher combination:
    #                  915 flop in 2D, 1371 flop in 3D (a third per stage kernel)
    #   whole step     populations in and out + c in and out: 80 B (2D), 160 B (3D)
    # FP32 peak: SMs x 128 lanes x 2 flop (FMA) x the sampled SM clock.
    dim = len(wl.shape)
    es = 8 if fp64 else 4
    lbm_B = 2 * (9 if dim == 2 else 19) * es + es + (es if wl.sugar else 0)  # + S in (sugar force)
    step_B = lbm_B + es + (es if wl.sugar else 0)                               # + c out (+ S out)
    tr_flop = 915.0 if dim == 2 else 1371.0
    # scheme variants, same count on their own formulation: WENO3 21 flop per reconstruction
    # (two candidates, two indicators, weights, normalisation, combination) -> 327 flop; the
    # sign-upwind choice one WENO5 reconstruction per face (+ face velocity) -> 477 flop
    if wl.scheme.get("weno3"):
        tr_flop = 327.0
    elif wl.scheme.get("sign_split"):
        tr_flop = 477.0
    ncls = max(1, len(wl.class_vs))
    step_B += 2 * es * (ncls - 1)  # every class's c in and out
    flop_of = {"rk3_sweep2d": tr_flop, "rk3_sweep3d": tr_flop, "rk_stage1": tr_flop / 3,
               "rk_stage2": tr_flop / 3, "rk_stage3": tr_flop / 3}
    sms = sm_count(dev)
    fp32_peak = fp32_peak_tflops(clk, sms)
    # ncu traffic was captured on the plain 2D workload's kernels only
    if wl is workloads.MAIN_2D:
        ncu_traffic = {k: kernel_traffic(k) for k in NCU_TRAFFIC}
    elif wl is workloads.MAIN_3D:
        ncu_traffic = {k: kernel_traffic(k, NCU_TRAFFIC_3D) for k in NCU_TRAFFIC_3D}
    else:
        ncu_traffic = {}

    def avg_s(name):
        n_, t_ = stats[name]
        return t_ * 1e-3 / n_
    roofline = None
    if dominant in flop_of:
        achieved = flop_of[dominant] * wl.nodes / avg_s(dominant) / 1e12
        roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": fp32_peak,
                    "peak_source": f"derived: {sms} SM x 128 FP32 lanes x 2 x sampled SM clock",
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": ncu_traffic.get(dominant),
                    "alg_flop_per_node": flop_of[dominant]}
    elif dominant == "lbm_collide_stream":
        achieved = lbm_B * wl.nodes / avg_s(dominant) / 1e9
        roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                    "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": ncu_traffic.get(dominant), "alg_bytes_per_node": lbm_B}
    if roofline and roofline.get("traffic"):  # ncu DRAM bytes per launch over the live duration
        roofline["dram_gbs"] = roofline["traffic"] / avg_s(roofline["kernel"]) / 1e9
    lbm_roofline = None
    if "lbm_collide_stream" in stats:
        a_ = lbm_B * wl.nodes / avg_s("lbm_collide_stream") / 1e9
        tr_ = ncu_traffic.get("lbm_collide_stream")
        lbm_roofline = {"bound": "hbm", "kernel": "lbm_collide_stream", "achieved": a_, "peak": peak,
                        "unit": "GB/s", "frac": a_ / peak, "traffic": tr_,
                        "dram_gbs": tr_ / avg_s("lbm_collide_stream") / 1e9 if tr_ else None,
                        "alg_bytes_per_node": lbm_B}
    if fp64:  # the L2-resident FP64 parity case: launch-bound, no roofline claim
        roofline = {"bound": None, "note": "2.4 MB working set in L2: launch-bound parity case, no roofline claim"}
    # the transport as a whole (one fused kernel or three stage kernels) against the FP32 peak
    tr_kernels = [k for k in ("rk3_sweep2d", "rk_stage1", "rk_stage2", "rk_stage3") if k in stats]
    transport_roofline = None
    if tr_kernels:
        t_tr = sum(avg_s(k) for k in tr_kernels)
        a_ = tr_flop * wl.nodes / t_tr / 1e12
        transport_roofline = {"bound": "alu", "kernels": tr_kernels, "achieved": a_, "peak": fp32_peak,
                              "unit": "TFLOP/s", "frac": a_ / fp32_peak, "alg_flop_per_node": tr_flop,
                              "us_per_step": t_tr * 1e6 * ncls}
        if ncls > 1:
            transport_roofline["note"] = f"per class; the three stage kernels run once per class ({ncls})"
    step_roofline = {"bound": "hbm", "alg_bytes_per_node": step_B,
                     "achieved": step_B * wl.nodes / (step_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": step_B * wl.nodes / (step_ms * 1e-3) / 1e9 / peak}
    if roofline and roofline.get("bound"):  # the whole coupled step beside the dominant kernel
        roofline["step_frac"] = step_roofline["frac"]
        roofline["step_achieved_gbs"] = step_roofline["achieved"]
        roofline["step_alg_bytes_per_node"] = step_B

    # ---- end to end through the C ABI with host buffers: H2D of c0 (pinned), init,
    # K steps, deposit read and D2H of the final c field, all inside the timed region
    c_host = torch.from_numpy(c0).pin_memory()
    c_out = torch.empty_like(c_host).pin_memory()
    S_host = torch.from_numpy(S0).pin_memory() if S0 is not None else None
    cls_host = [torch.from_numpy(a.astype(np_dt)).pin_memory() for a in wl.initial_classes()] if wl.class_vs else []
    sim2 = lw.Simulation(wl.shape, fp64=fp64, stream=stream, **kw)
    sim2.init(c_host)
    if S_host is not None:
        sim2.set_sugar(S_host)
    for k, ck in enumerate(cls_host):
        sim2.set_class(k, ck)
    sim2.step(1)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    sim2.init(c_host)
    if S_host is not None:
        sim2.set_sugar(S_host)
    for k, ck in enumerate(cls_host):
        sim2.set_class(k, ck)
    sim2.step(args.steps)
    dep = sim2.deposit
    lw.lbm_wenoc_fields(sim2.handle, None, None, c_out)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = job_time_ms(e2e_s * 1e3, device=dev) * 1e-3
    e2e = {"value": world * wl.nodes * args.steps / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": (c_host.numel() * c_host.element_size() * (2 if S_host is not None else 1)
                                  + sum(t.numel() * t.element_size() for t in cls_host)) / args.steps,
           "d2h_bytes_per_step": (c_out.numel() * c_out.element_size() + 8) / args.steps,
           "note": "per job: H2D c0 (+ S0) + init + K steps + deposit (8 B) + D2H c, host wall clock"}
    assert np.isfinite(dep)
    sim2.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, dt = run_oracle_sample(wl, args.cpu_steps, threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"FP64 C oracle, {'x'.join(map(str, wl.shape[:-1]))}x"
                         f"{wl.shape[-1] if len(wl.shape) == 2 else 64} lattice, "
                         f"{args.cpu_steps} steps after 1 warm-up ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32", "data": "synthetic",
            "config": {"workload": wl.name, "shape": list(wl.shape), "lattice": LATTICE,
                       "tau": wl.tau, "A": wl.gravity * wl.density_contrast, "Vs": wl.settling_velocity,
                       "kappa": wl.diffusivity, "parallelism": f"replicas{world}", **({"sugar": wl.sugar} if wl.sugar else {}),
                       **({"scheme": wl.scheme} if wl.scheme else {}),
                       **({"class_vs": list(wl.class_vs)} if wl.class_vs else {}),
                       "l2": (lambda mb: f"inputs larger than L2 (populations {mb:.0f} MB)" if mb > 129
                              else f"inputs fit in L2 (populations {mb:.1f} MB): no L2 flush claim")(
                           wl.nodes * (9 if len(wl.shape) == 2 else 19) * (8 if fp64 else 4) / 1e6)},
            "roofline": roofline, "lbm_roofline": lbm_roofline, "transport_roofline": transport_roofline,
            "step_roofline": step_roofline,
            "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()


def bench_batch(args):
    """64 independent 2D instances (sizes and parameters of workloads.batch_sweep) advanced
    by the persistent launch (per-size segment heights from the autotuner), against the same
    batch with one launch per kernel type and step, and against the instances run one after
    the other on the same GPU (each for the same number of steps)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2106_07694_gb300 import build as lbuild
    lbuild.build()
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    wls = workloads.batch_sweep(64)
    specs = [dict(shape=w.shape, **phys_kwargs(w)) for w in wls]
    nodes = sum(w.nodes for w in wls)
    b = lw.Batch(specs)
    b.set_persistent(BATCH_MODE)
    rows = b.autotune(8)
    for inst, w in zip(b.instances, wls):
        inst.init(torch.from_numpy(w.initial_c().astype(np.float32)).cuda())
    b.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = lw.lbm_wenoc_batch_launch_count(b.handle)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = lw.lbm_wenoc_batch_launch_count(b.handle) - l0
    if b.status() != lw.LW_OK:
        raise RuntimeError("device status set in the batched run")
    value = nodes * args.steps / (ms * 1e-3) / 1e9
    # the same batch in the other launch forms: all phases persistent (one launch per 16
    # steps), split (grouped fluid launch + persistent stage launch per step), grouped
    other_ms = {}
    for mode in (1, 2, 0):
        if mode == BATCH_MODE:
            continue
        b.set_persistent(mode)
        b.step(args.warmup)
        torch.cuda.synchronize()
        e0.record()
        b.step(args.steps)
        e1.record()
        torch.cuda.synchronize()
        other_ms[mode] = e0.elapsed_time(e1)
        if b.status() != lw.LW_OK:
            raise RuntimeError(f"device status set in the batched run of form {mode}")
    b.close()
    grouped_ms = other_ms[0]
    # sequential: the same instances one after the other, same number of steps each
    seq_ms = 0.0
    for w, sp in zip(wls, specs):
        s = lw.Simulation(w.shape, **{k: v for k, v in sp.items() if k != "shape"})
        s.init(torch.from_numpy(w.initial_c().astype(np.float32)).cuda())
        s.step(args.warmup)
        torch.cuda.synchronize()
        e0.record()
        s.step(args.steps)
        e1.record()
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)
        s.close()
    seq = nodes * args.steps / (seq_ms * 1e-3) / 1e9
    peak, _ = load_peaks()
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch_sweep_64_d2q9_f32", "instances": len(wls), "nodes": nodes,
                   "autotuned_segment_rows": rows, "seed": 0},
        "sequential": {"value": seq, "unit": UNIT, "ms_per_step": seq_ms / args.steps,
                       "note": "each instance alone through lbm_wenoc_step, one after the other"},
        "grouped": {"value": nodes * args.steps / (grouped_ms * 1e-3) / 1e9, "unit": UNIT,
                    "ms_per_step": grouped_ms / args.steps,
                    "note": "same batch, one launch per kernel type and step instead of the persistent launch"},
        "launch_form": BATCH_FORMS[BATCH_MODE],
        "other_forms": {BATCH_FORMS[m]: {"value": nodes * args.steps / (t_ * 1e-3) / 1e9, "unit": UNIT,
                                         "ms_per_step": t_ / args.steps} for m, t_ in other_ms.items()},
        "batched_over_sequential": value / seq,
        "step_roofline": {"bound": "hbm", "alg_bytes_per_node": 80, "achieved": 80 * value, "peak": peak,
                          "unit": "GB/s", "frac": 80 * value / peak},
        "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def bench_adjoint(args):
    """Reverse-mode gradient of the deposited mass on the 512 x 1024 lattice (2000 steps,
    state kept every 100): time of one lbm_wenoc_deposit_gradient call (forward with
    checkpoints, per-segment recompute, reverse sweep) against the plain forward of the
    same steps.  GLUPS = nodes x steps / gradient time.  e2e: the torch.autograd path
    from a pinned host c0 to dJ/dc0 back in host memory."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2106_07694_gb300 import build as lbuild
    lbuild.build()
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.autograd import deposited_mass
    wl = workloads.ADJOINT_2D
    # the gradient is defined over the whole 2000-step horizon; the overrides only serve
    # small profiling captures
    nsteps = args.adjoint_steps or wl.steps
    seg = args.adjoint_segment or wl.extra["segment"]
    kw = dict(phys_kwargs(wl), lf_alpha=wl.extra["lf_alpha"])
    c0 = torch.from_numpy(wl.initial_c().astype(np.float32)).cuda()
    sim = lw.Simulation(wl.shape, **kw)
    nbytes = lw.lbm_wenoc_gradient_workspace_bytes(sim.params, nsteps, seg)
    adj = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    grad = torch.empty(c0.shape, dtype=torch.float32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):  # forward alone
        sim.init(c0)
        sim.step(nsteps)
    torch.cuda.synchronize()
    e0.record()
    sim.init(c0)
    sim.step(nsteps)
    e1.record()
    J_fwd = sim.deposit
    fwd_ms = e0.elapsed_time(e1)
    lw.lbm_wenoc_deposit_gradient(sim.handle, c0, nsteps, seg, adj, nbytes, grad)  # warm-up
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = lw.lbm_wenoc_launch_count(sim.handle)
    e0.record()
    J, dvs = lw.lbm_wenoc_deposit_gradient(sim.handle, c0, nsteps, seg, adj, nbytes, grad)
    e1.record()
    torch.cuda.synchronize()
    grad_ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = lw.lbm_wenoc_launch_count(sim.handle) - l0
    if J != J_fwd:
        raise RuntimeError("forward of the gradient call differs from the plain forward")
    # e2e through autograd: pinned host c0 in, dJ/dc0 back to pinned host memory
    host_c0 = c0.cpu().pin_memory()
    host_g = torch.empty(c0.shape, dtype=torch.float32).pin_memory()
    kw2 = {k: v for k, v in kw.items() if k != "settling_velocity"}

    def e2e_call():
        x = host_c0.cuda(non_blocking=True).requires_grad_(True)
        vs = torch.tensor(wl.settling_velocity, dtype=torch.float64, requires_grad=True)
        out = deposited_mass(x, vs, nsteps, wl.shape, segment=seg, **kw2)
        out.backward()
        host_g.copy_(x.grad, non_blocking=True)
        torch.cuda.synchronize()

    e2e_call()  # warm-up: the wrapper allocates its handle and workspace once
    t0 = time.perf_counter()
    e2e_call()
    e2e_s = time.perf_counter() - t0
    # the same gradient with every step recorded in HBM (no checkpoints, no recompute)
    nb_all = lw.lbm_wenoc_gradient_workspace_bytes(sim.params, nsteps, nsteps)
    adj_all = torch.empty(nb_all, dtype=torch.uint8, device="cuda")
    lw.lbm_wenoc_deposit_gradient(sim.handle, c0, nsteps, nsteps, adj_all, nb_all, grad)
    torch.cuda.synchronize()
    e0.record()
    J_all, dvs_all = lw.lbm_wenoc_deposit_gradient(sim.handle, c0, nsteps, nsteps, adj_all, nb_all, grad)
    e1.record()
    torch.cuda.synchronize()
    all_ms = e0.elapsed_time(e1)
    del adj_all
    # per-kernel averages: one more gradient call with an event pair around every launch
    lw.lbm_wenoc_profile_enable(sim.handle, True)
    lw.lbm_wenoc_profile_read(sim.handle, reset=True)
    lw.lbm_wenoc_deposit_gradient(sim.handle, c0, nsteps, seg, adj, nbytes, grad)
    prof = lw.lbm_wenoc_profile_read(sim.handle, reset=True)
    lw.lbm_wenoc_profile_enable(sim.handle, False)
    kernels = {k: {"launches": c, "avg_us": 1e3 * ms / c, "total_ms": ms} for k, (c, ms) in prof.items() if c}
    nodes = wl.nodes
    peak_alu = fp32_peak_tflops(clk)
    faces_us = kernels.get("adj_faces", {}).get("avg_us")
    value = nodes * nsteps / (grad_ms * 1e-3) / 1e9
    line = {
        "metric": ADJOINT_METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": nsteps,
        "warmup": args.warmup, "ms_per_step": grad_ms / nsteps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "nodes": nodes, "segment": seg, "lf_alpha": kw["lf_alpha"],
                   "adjoint_workspace_bytes": nbytes, "l2": "working set > L2 (states of one segment)"},
        "forward": {"ms": fwd_ms, "glups": nodes * nsteps / (fwd_ms * 1e-3) / 1e9},
        "gradient_over_forward": grad_ms / fwd_ms,
        "no_recompute": {"ms_per_step": all_ms / nsteps, "gradient_over_forward": all_ms / fwd_ms,
                         "adjoint_workspace_bytes": nb_all, "same_result": bool(J_all == J and dvs_all == dvs),
                         "note": "all step records kept in HBM instead of a checkpoint every 100 steps"},
        "J": J, "dJ_dVs": dvs, "grad_l2": float(torch.linalg.vector_norm(grad.double())),
        "kernels": kernels,
        "roofline": None if not faces_us else {
            "kernel": "adj_faces", "bound": "alu", "alg_flop_per_node": ADJ_FACES_FLOP,
            "achieved": ADJ_FACES_FLOP * nodes / (faces_us * 1e-6) / 1e12, "peak": peak_alu,
            "unit": "TFLOP/s", "frac": ADJ_FACES_FLOP * nodes / (faces_us * 1e-6) / 1e12 / peak_alu,
            "peak_source": f"derived: {sm_count()} SM x 128 FP32 lanes x 2 x sampled SM clock",
            "traffic": kernel_traffic("adj_faces")},
        "e2e": {"value": nodes * nsteps / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": 4 * nodes / nsteps,
                "d2h_bytes_per_step": (4 * nodes + 8) / nsteps},
        "gpu_launches": int(launches), "clocks": clk,
    }
    sim.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=0, help="override the horizon (profiling only)")
    ap.add_argument("--adjoint-segment", type=int, default=0, help="override the checkpoint spacing")
    ap.add_argument("--workload", default="2d", choices=sorted(WORKLOADS) + ["batch", "adjoint"],
                    help="2d: the 2048x4096 D2Q9 case the metric is quoted on; 3d: 256x256x512 D3Q19; "
                         "sugar: the 2048x4096 case with the sugar scalar; batch; adjoint")
    ap.add_argument("--lattice", default="",
                    help="override the lattice, e.g. 256x256x128 (profiling captures of a smaller case only; "
                         "the line then names the smaller lattice)")
    args = ap.parse_args()
    global WL, METRIC, LATTICE
    if args.workload == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched sweep has no oracle arm; "
                              "the oracle is timed on the single-instance workloads"}))
            return
        bench_batch(args)
        return
    if args.workload == "adjoint":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the gradient has no oracle arm; "
                              "the oracle is timed on the single-instance workloads"}))
            return
        bench_adjoint(args)
        return
    WL, METRIC, LATTICE = WORKLOADS[args.workload]
    if args.lattice:
        shape = tuple(int(v) for v in args.lattice.lower().split("x"))
        if len(shape) != len(WL.shape):
            ap.error("--lattice needs as many extents as the workload's lattice")
        WL = WL.with_(shape=shape, name=f"{WL.name}_as_{args.lattice}")
        METRIC = METRIC + f" [lattice {args.lattice}]"
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
