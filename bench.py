"""FEWHA benchmark: ELT frame latency p50/p99 (us) and PCG iterations/s on one
B300, FP32 fused-graph path beside the plain FP64 path, on synthetic
von Karman frames of the ELT bulk configuration (D = 39 m, 6 LGS, 84x84
subapertures, 9 layers on 128^2 grids, db3 with 4 levels, 4 warm-started PCG
iterations per frame).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fewha|reference]

A step is one frame of Alg. 1 up to the layers: slopes in -> RHS -> warm
restart (residual replacement every 10 frames) -> 4 iterations of Alg. 2 ->
layers phi = W^T c out.  Prints one JSON line (rank 0).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2009_00946_b300 import configs, synth  # noqa: E402

METRIC = "ELT frame latency p50/p99 µs & PCG iter/s, FP32-graph vs plain FP64 on B300"
UNIT = "us"
N_ITER = 4
K_RR = 10
L2_FLUSH_BYTES = 512 << 20


def workload_config():
    return configs.c2_elt()


def config_block(cfg, extra=None):
    d = {"workload": "ELT MCAO bulk: D=39 m, 6 LGS (90 km) on a 1-arcmin-radius hexagon, 84x84 subapertures, "
                     "9 layers 0-16 km on 128^2 grids, db3 J=4, 4 warm-started PCG iterations per frame, "
                     "residual replacement every 10 frames",
         "frames": "synthetic von Karman frozen flow (r0=0.157 m, L0=25 m), 500 Hz, sigma=0.1 rad",
         "n_coeff": sum(l["n"] ** 2 for l in cfg["layers"]),
         "n_slopes": sum(2 * w["n_sub"] ** 2 for w in cfg["wfs"]),
         "l2": "flushed between timed frames (512 MiB write, untimed)"}
    if extra:
        d.update(extra)
    return d


def algorithmic_bytes_per_frame(cfg, n_iter, elem=4):
    """Per PCG iteration 16N + 4 NW elements (each operator reads its input and
    writes its output once: inverse DWT 2N, P N+NW, Gamma/C/Gamma^T 2NW,
    P^T NW+N, forward DWT + alpha D z 3N, update 9N); per frame add the RHS
    and restart S + 2NW + 8N and the layers output 2N."""
    N = sum(l["n"] ** 2 for l in cfg["layers"])
    NW = sum((w["n_sub"] + 1) ** 2 for w in cfg["wfs"])
    S = sum(2 * w["n_sub"] ** 2 for w in cfg["wfs"])
    return elem * (n_iter * (16 * N + 4 * NW) + S + 2 * NW + 10 * N)


def algorithmic_bytes_per_iteration(cfg, elem=4):
    """16N + 4 NW elements: one PCG iteration of Alg. 2 with its operator M."""
    N = sum(l["n"] ** 2 for l in cfg["layers"])
    NW = sum((w["n_sub"] + 1) ** 2 for w in cfg["wfs"])
    return elem * (16 * N + 4 * NW)


def roofline_block(cfg, t_launch_us, per_iter_us, l2, hbm, hbm_kind, traffic):
    """Roofline of the fused frame kernel against the measured L2 bandwidth
    (its working set stays in L2), with the HBM figure beside it.
    t_launch_us: event-timed duration of one 4-iteration solve launch;
    per_iter_us: marginal cost of one PCG iteration; l2: measure_l2() result
    (the larger of the read and the copy figure is the peak)."""
    alg = algorithmic_bytes_per_frame(cfg, N_ITER)
    it_bytes = algorithmic_bytes_per_iteration(cfg)
    achieved = alg / (t_launch_us * 1e-6) / 1e9
    l2_peak = max(l2["read_gbs"], l2["copy_gbs"])
    it_ach = it_bytes / (per_iter_us * 1e-6) / 1e9 if per_iter_us and per_iter_us > 0 else None
    return {"bound": "l2", "achieved": achieved, "peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
            "traffic": traffic,
            "traffic_note": "DRAM bytes per launch, ncu full capture (cold caches); the L2 keeps the state, so "
                            "traffic is far below the algorithmic bytes",
            "kernel": "k_fused_frame", "duration_us": t_launch_us, "algorithmic_bytes": alg,
            "peak_kind": "of measured (fewha_measure_l2 in this run: %d MiB resident buffer, %d passes per "
                         "launch, fastest of %d; read %.0f GB/s, copy read+write %.0f GB/s; the larger is the "
                         "peak)" % (l2["bytes"] >> 20, l2["passes"], l2["reps"], l2["read_gbs"], l2["copy_gbs"]),
            "per_iteration": {"algorithmic_bytes": it_bytes, "us": per_iter_us, "achieved": it_ach,
                              "frac": it_ach / l2_peak if it_ach else None,
                              "what": "16N + 4NW FP32 elements per PCG iteration / marginal iteration time"},
            "hbm": {"peak": hbm, "frac": achieved / hbm, "peak_kind": hbm_kind}}


def slope_pool(cfg, count, seed=None):
    atm = synth.Atmosphere(cfg, seed)
    return np.stack([atm.slopes(k) for k in range(count)]).astype(np.float32)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 20):
        self.cmd = ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                    "--format=csv,noheader,nounits", "-lms", str(period_ms)]
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_latency(cfg, n_frames, pool_np, keep=None):
    """The FP64 CPU oracle as it stands, one host core: per-frame latency (us).
    With keep (a list) the layers of every frame are appended to it."""
    from oracle import fewha_oracle as fo
    R = fo.Reconstructor(cfg)
    times = []
    for k in range(n_frames):
        s = pool_np[k % len(pool_np)].astype(np.float64)
        t0 = time.perf_counter()
        R.frame(s, N_ITER, warm=True, k_rr=K_RR)
        lay = R.layers()
        times.append((time.perf_counter() - t0) * 1e6)
        if keep is not None:
            keep.append(lay)
    return times


def _oracle_stream(args):
    """One worker of the all-core baseline: the unmodified oracle over its own
    frozen-flow frames (its own seed), per-frame latencies (us)."""
    cfg, seed, n = args
    pool = slope_pool(cfg, n, seed=seed)
    return cpu_oracle_latency(cfg, n, pool)


def cpu_oracle_all_cores(cfg, frames_per_core=6):
    """The oracle on every host core at once: one independent frame stream per
    core (spawned processes, each the unmodified one-thread oracle), wall time
    of the whole, aggregate frames per second.  The oracle's per-frame work is
    not split over layers or sensors: its numpy operators on 128^2 layers are
    too small for threads (the interpreter lock serialises them) or for
    process fan-out (each task would move about 1 MB for 5 ms of work)."""
    import multiprocessing as mp
    cores = max(1, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    jobs = [(cfg, int(cfg["seed"]) + 1000 + i, frames_per_core) for i in range(cores)]
    # one thread per process (the children inherit the environment)
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        t0 = time.perf_counter()
        with ctx.Pool(cores) as p:
            res = p.map(_oracle_stream, jobs)
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    lat = [x for r in res for x in r[1:]]   # first frame of each stream: warm-up
    return {"frames_per_s": cores * frames_per_core / wall, "wall_s": wall, "cores": cores,
            "per_frame_p50_us": float(np.percentile(lat, 50)), "kind": "oracle",
            "sample": "%d independent streams x %d ELT frames (one per host core, spawned processes; process "
                      "start and frame synthesis inside the wall time)" % (cores, frames_per_core)}


def parity_vs_oracle(fewha, cfg, pool, oracle_layers):
    """The same frames through a fresh FP32 fused handle (host buffers, one
    graph per frame): relative L2 error of the layers against the oracle's."""
    S = fewha.Solver(cfg, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR)
    out = np.empty(S.N, np.float32)
    errs = []
    for k, ref in enumerate(oracle_layers):
        S.frame(pool[k % len(pool)], N_ITER, warm=True, layers_out=out)
        errs.append(float(np.linalg.norm(out.astype(np.float64) - ref) / np.linalg.norm(ref)))
    S.close()
    return {"layers_rel_l2_max": max(errs), "layers_rel_l2_median": float(np.median(errs)), "frames": len(errs),
            "tolerance": 1e-4, "against": "FP64 CPU oracle on the same frames (the cpu_baseline run), "
                                          "warm-started, residual replacement every 10 frames"}


# DRAM bytes (read + write) of one k_fused_frame launch on this workload from
# the committed full ncu capture, valid only for the kernel source it was
# taken on (sha256 prefix of csrc/fused.cu + csrc/fused_cascade.cuh); any
# other source reports null.
NCU_TRAFFIC = {"fused_cu_sha256": "5d9850da7f073d22", "dram_bytes": 5646336,
               "summary": "profiles/k_fused_frame_elt_full.md"}


def fused_source_sha():
    """sha256 of the fused frame kernel's sources (fused.cu + fused_cascade.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("fused.cu", "fused_cascade.cuh"):
        with open(os.path.join(ROOT, "paper_2009_00946_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def fused_traffic():
    sha = fused_source_sha()
    return NCU_TRAFFIC["dram_bytes"] if sha.startswith(NCU_TRAFFIC["fused_cu_sha256"]) else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6400.0, "of fallback (6.4 TB/s; no MEASURED_PEAKS.json)"


def run_reference(args):
    """Reference arm: the CPU oracle (there is no runnable reference code)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload_config()
    n_time = min(args.steps, 40)
    n_warm = min(args.warmup, 3)
    pool = slope_pool(cfg, n_time + n_warm)
    t = cpu_oracle_latency(cfg, n_time + n_warm, pool)[n_warm:]
    p50 = float(np.percentile(t, 50))
    line = {"impl": "reference", "metric": METRIC, "value": p50, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(t)) / 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(cfg),
            "p99_us": float(np.percentile(t, 99)),
            "cpu_baseline": {"value": p50, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d frames of the workload after %d warm-up frames (of the %d requested)"
                                       % (n_time, n_warm, args.steps)},
            "e2e": {"value": p50, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_frames(S, torch, pool_dev, start, K, layers_dev, flush, events=True):
    """K frames through the device-pointer graph, L2 flushed before each."""
    st = S.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        with torch.cuda.stream(st):
            flush.fill_(float(k & 7))
        ev[k][0].record(st)
        S.frame(pool_dev[(start + k) % pool_dev.shape[0]], N_ITER, warm=True, layers_out=layers_dev)
        ev[k][1].record(st)
    st.synchronize()
    return [a.elapsed_time(b) * 1e3 for a, b in ev]


def time_solve(S, torch, n_iter, K, flush):
    """Average duration (us) of one solve launch (RHS + restart + n_iter iterations)."""
    st = S.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        with torch.cuda.stream(st):
            flush.fill_(1.0)
        ev[k][0].record(st)
        S.solve(n_iter, warm=True)
        ev[k][1].record(st)
    st.synchronize()
    S.sync()
    return float(np.mean([a.elapsed_time(b) * 1e3 for a, b in ev]))


def bench_elt_dm_frame(torch, fewha, dev, flush, n_frames):
    """35-layer ELT frame with the least-squares fit onto 3 mirrors (the whole
    of Alg. 1 as one captured graph): latency p50/p99 (us), device buffers."""
    cfg = configs.c3_elt_dm()
    pool = torch.from_numpy(slope_pool(cfg, 16)).to(dev)
    S = fewha.Solver(cfg, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR)
    lay = torch.empty(S.N, dtype=torch.float32, device=dev)
    dm = torch.empty(S.NA, dtype=torch.float32, device=dev)
    st = S.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
    for k in range(5):
        S.frame(pool[k % 16], N_ITER, warm=True, gain=cfg["gain"], n_fit=cfg["n_fit"], layers_out=lay, dm_out=dm)
    S.sync()
    tuned = S.autotune(N_ITER, 5)   # once at start-up: the cluster shape that is fastest for 35 layers
    for k in range(5):
        S.frame(pool[k % 16], N_ITER, warm=True, gain=cfg["gain"], n_fit=cfg["n_fit"], layers_out=lay, dm_out=dm)
    for k in range(n_frames):
        with torch.cuda.stream(st):
            flush.fill_(float(k & 7))
        ev[k][0].record(st)
        S.frame(pool[k % 16], N_ITER, warm=True, gain=cfg["gain"], n_fit=cfg["n_fit"], layers_out=lay, dm_out=dm)
        ev[k][1].record(st)
    st.synchronize()
    S.sync()
    t = [a.elapsed_time(b) * 1e3 for a, b in ev]
    out = {"workload": "ELT with 35 layers 0-25 km (128^2, J=4), 4 iterations, least-squares fit (8 CG steps, "
                       "5x5 directions) onto 3 mirrors at 0/4/12.7 km, gain 1",
           "p50_us": float(np.percentile(t, 50)), "p99_us": float(np.percentile(t, 99)), "frames": n_frames,
           "n_coeff": S.N, "n_act": S.NA, "plan": S.describe(), "autotune": tuned}
    S.close()
    return out


def bench_maory_frame(torch, fewha, dev, flush, n_frames):
    """The paper's own timing case (Sec. 4.1, Table 2; L = M = 6, 4 iterations):
    whole frame with the co-located fit through one graph, device buffers."""
    cfg = configs.maory(6, N_ITER)
    cfg["lgs_tip_tilt_filter"] = True   # laser guide stars do not sense tip/tilt (the NGS do)
    pool = torch.from_numpy(slope_pool(cfg, 16)).to(dev)
    S = fewha.Solver(cfg, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR)
    lay = torch.empty(S.N, dtype=torch.float32, device=dev)
    dm = torch.empty(S.NA, dtype=torch.float32, device=dev)
    st = S.stream
    for k in range(5):
        S.frame(pool[k % 16], N_ITER, warm=True, gain=cfg["gain"], layers_out=lay, dm_out=dm)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
    for k in range(n_frames):
        with torch.cuda.stream(st):
            flush.fill_(float(k & 7))
        ev[k][0].record(st)
        S.frame(pool[k % 16], N_ITER, warm=True, gain=cfg["gain"], layers_out=lay, dm_out=dm)
        ev[k][1].record(st)
    st.synchronize()
    S.sync()
    t = [a.elapsed_time(b) * 1e3 for a, b in ev]
    out = {"workload": "MAORY-like (Sec. 4.1 / Table 2): D=39 m, 6 LGS 80x80 (tip-tilt filtered) + NGS tip-tilt "
                       "2x2/1x1/1x1, L = M = 6 layers/mirrors (0-20 km, 128^2, J=4; 81^2/48^2/54^2 actuators), "
                       "4 iterations, co-located fit, gain 0.5",
           "p50_us": float(np.percentile(t, 50)), "p99_us": float(np.percentile(t, 99)), "frames": n_frames,
           "paper_context": "paper (Sec. 4.3): about 3 ms per reconstruction on 2x 8-core Haswell (CPU), 8.6 ms on "
                            "a V100; other hardware, context only",
           "plan": S.describe()}
    S.close()
    return out


def bench_mode_frame(torch, fewha, dev, flush, n_frames, mode):
    """The MAORY-like asterism and layers in the LTAO or MOAO operating mode
    (Sec. 4.3 times LTAO, MOAO and MCAO): whole frame with the least-squares
    mirror fit (8 CG steps) through one graph, device buffers, open loop."""
    cfg = configs.maory_mode(mode)
    pool = torch.from_numpy(slope_pool(cfg, 16)).to(dev)
    S = fewha.Solver(cfg, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR)
    lay = torch.empty(S.N, dtype=torch.float32, device=dev)
    dm = torch.empty(S.NA, dtype=torch.float32, device=dev)
    st = S.stream
    for k in range(5):
        S.frame(pool[k % 16], N_ITER, warm=True, gain=cfg["gain"], n_fit=cfg["n_fit"], layers_out=lay, dm_out=dm)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
    for k in range(n_frames):
        with torch.cuda.stream(st):
            flush.fill_(float(k & 7))
        ev[k][0].record(st)
        S.frame(pool[k % 16], N_ITER, warm=True, gain=cfg["gain"], n_fit=cfg["n_fit"], layers_out=lay, dm_out=dm)
        ev[k][1].record(st)
    st.synchronize()
    S.sync()
    t = [a.elapsed_time(b) * 1e3 for a, b in ev]
    what = ("one ground mirror (81^2) fitted on axis" if mode == "ltao" else
            "%d objects on the 5x5 grid, one ground mirror (81^2) each" % len(cfg["dms"]))
    out = {"workload": "MAORY-like asterism and layers (6 LGS 80x80 + 3 tip-tilt NGS, 6 layers 0-20 km, 128^2, "
                       "J=4), %s, %s, 4 iterations + 8 fitting CG steps, open loop" % (mode.upper(), what),
           "p50_us": float(np.percentile(t, 50)), "p99_us": float(np.percentile(t, 99)), "frames": n_frames,
           "plan": S.describe()}
    S.close()
    return out


def bench_autograd(torch, fewha, dev, flush, reps=20):
    """The differentiable solve on the autograd configuration (D = 16 m, 4 LGS
    40x40, 5 layers 64^2, J = 3, 4 cold-start iterations): a batch of 32
    frames, taped forward and reverse mode (gradients in gamma, alpha, w and
    the slopes), FP32 vectors with FP64 scalars and in FP64; the frame batch
    in one launch sequence against the same frames one call each."""
    from paper_2009_00946_b300 import synth
    cfg = configs.c5_autograd()
    B = 32
    S_np, T_np = synth.frames(cfg, B)
    out = {"workload": "autograd configuration: D=16 m, 4 LGS (90 km) at 60 arcsec, 40x40 subapertures, 5 layers "
                       "64^2 (J=3), 4 cold-start PCG iterations, batch of 32 frames, loss sum |phi - phi_true|^2",
           "frames": B}
    for name, prec, dt in (("fp32", fewha.FP32, torch.float32), ("fp64", fewha.FP64, torch.float64)):
        S = fewha.Solver(cfg, precision=prec)
        st = S.stream
        with torch.cuda.stream(st):
            sd = torch.from_numpy(S_np).to(dev, dt).contiguous()
            phit = torch.from_numpy(T_np.reshape(B, -1)).to(dev, dt)
            tape = torch.empty(S.tape_bytes_batch(N_ITER, B), dtype=torch.uint8, device=dev)
            tapes1 = [torch.empty(S.tape_bytes(N_ITER), dtype=torch.uint8, device=dev) for _ in range(B)]
            phi = torch.empty(B, S.N, dtype=dt, device=dev)
            gg = torch.empty(B, S.n_layers, dtype=torch.float64, device=dev)
            ga = torch.empty(B, dtype=torch.float64, device=dev)
            gw = torch.empty(B, S.n_wfs, dtype=torch.float64, device=dev)
            gs = torch.empty_like(sd)
        st.synchronize()

        def fwd_batch():
            S.solve_taped_batch(sd, N_ITER, tape, phi)

        def bwd_batch():
            S.backward_batch(sd, N_ITER, tape, phibar, gg, ga, gw, gs)

        def fwd_loop():
            for b in range(B):
                S.solve_taped(sd[b], N_ITER, tapes1[b], phi[b])

        def bwd_loop():
            for b in range(B):
                S.backward(sd[b], N_ITER, tapes1[b], phibar[b], gg[b], ga[b:b + 1], gw[b], gs[b])

        def timed(fn):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for k in range(reps):
                with torch.cuda.stream(st):
                    flush.fill_(float(k & 7))
                ev[k][0].record(st)
                fn()
                ev[k][1].record(st)
            st.synchronize()
            return float(np.percentile([a.elapsed_time(b) * 1e3 for a, b in ev], 50))

        fwd_batch()
        with torch.cuda.stream(st):
            phibar = (2.0 * (phi - phit)).contiguous()
        st.synchronize()
        for fn in (bwd_batch, fwd_loop, bwd_loop):
            fn()
        st.synchronize()
        n0 = S.launch_count()
        fwd_batch()
        bwd_batch()
        st.synchronize()
        launches = S.launch_count() - n0
        rec = {"forward_us": timed(fwd_batch), "backward_us": timed(bwd_batch),
               "one_call_per_frame_forward_us": timed(fwd_loop), "one_call_per_frame_backward_us": timed(bwd_loop),
               "kernel_launches_forward_and_backward": launches}
        rec["speedup_forward_and_backward"] = ((rec["one_call_per_frame_forward_us"] +
                                                rec["one_call_per_frame_backward_us"]) /
                                               (rec["forward_us"] + rec["backward_us"]))
        S.sync()
        out[name] = rec
        S.close()
    out["how"] = ("CUDA events around fewha_solve_taped_batch / fewha_backward_batch on the solver's stream, device "
                  "tensors, L2 flushed before each, median of %d; the one-call-per-frame lines run the same frames "
                  "through fewha_solve_taped / fewha_backward one frame at a time" % reps)
    return out


def bench_batch(torch, fewha, dev, flush, n_frames):
    """64 uneven instances advanced by one fused launch per group (the
    autotuner's grouping by layer size) per frame, against the
    same 64 instances solved one after another on the plain FP64 path and one
    fused FP32 launch each (one frame graph per instance, back to back)."""
    cfgs = configs.c4_batch(64)
    per = [synth.random_slopes(c, 7).astype(np.float32) for c in cfgs]
    B = fewha.Batch(cfgs, k_rr=K_RR)
    s = torch.from_numpy(B.concat_slopes(per)).to(dev)
    lay = torch.empty(B.N, dtype=torch.float32, device=dev)
    st = B.stream
    for _ in range(5):
        B.frame(s, N_ITER, True, lay)

    def timed():
        for _ in range(3):
            B.frame(s, N_ITER, True, lay)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
        for k in range(n_frames):
            with torch.cuda.stream(st):
                flush.fill_(float(k & 7))
            ev[k][0].record(st)
            B.frame(s, N_ITER, True, lay)
            ev[k][1].record(st)
        st.synchronize()
        B.sync()
        return [a.elapsed_time(b) * 1e3 for a, b in ev]

    # once at start-up: the whole batch in one launch (cluster shape and
    # sensor-tile bound tuned), then any grouping by layer size
    B.set_max_launches(1)
    tuned1 = B.autotune(N_ITER, 3)
    t1 = timed()
    plan1 = B.describe()
    B.set_max_launches(0)
    tuned = B.autotune(N_ITER, 3)
    t = timed()
    p50 = float(np.percentile(t, 50))
    p50_1 = float(np.percentile(t1, 50))
    alg = sum(algorithmic_bytes_per_frame(c, N_ITER) for c in cfgs)
    plan = B.describe()
    N, S_tot = B.N, B.S
    B.close()
    # sequential: one plain FP64 handle per instance, solved one after another
    solvers = [fewha.Solver(c, precision=fewha.FP64, path=fewha.PATH_PLAIN, k_rr=K_RR) for c in cfgs]
    s64 = [torch.from_numpy(x.astype(np.float64)).to(dev) for x in per]
    reps = 3
    for S, x in zip(solvers, s64):
        S.set_frame(x)
        S.solve(N_ITER, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        for S, x in zip(solvers, s64):
            S.set_frame(x)
            S.solve(N_ITER, True)
        for S in solvers:
            S.sync()
    seq = (time.perf_counter() - t0) / reps * 1e6
    for S in solvers:
        S.close()
    # the same instances one fused FP32 launch each, back to back on one stream
    st1 = torch.cuda.Stream()
    solvers = [fewha.Solver(c, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR, stream=st1) for c in cfgs]
    s32 = [torch.from_numpy(x).to(dev) for x in per]
    l32 = [torch.empty(S.N, dtype=torch.float32, device=dev) for S in solvers]
    for S, x, y in zip(solvers, s32, l32):
        S.frame(x, N_ITER, warm=True, layers_out=y)
    ev1 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for k in range(5):
        with torch.cuda.stream(st1):
            flush.fill_(float(k & 7))
        ev1[k][0].record(st1)
        for S, x, y in zip(solvers, s32, l32):
            S.frame(x, N_ITER, warm=True, layers_out=y)
        ev1[k][1].record(st1)
    st1.synchronize()
    seq32 = float(np.percentile([a.elapsed_time(b) * 1e3 for a, b in ev1], 50))
    for S in solvers:
        S.sync()
        S.close()
    hbm, _ = measured_peaks()
    return {"workload": "64 independent instances: D 8-39 m, 16-84 subapertures, 2-9 layers on 32^2-256^2 grids, "
                        "3-6 LGS, 4 warm-started iterations each, FP32, one fused launch per group of instances "
                        "(the autotuner's grouping by layer size) per frame",
            "n_coeff": N, "n_slopes": S_tot, "p50_us": p50, "p99_us": float(np.percentile(t, 99)),
            "instance_frames_per_s": 64 * 1e6 / p50, "frames": n_frames, "autotune": tuned,
            "sequential_fp64_us": seq, "sequential_fp64_instance_frames_per_s": 64 * 1e6 / seq,
            "speedup_vs_sequential_fp64": seq / p50,
            "sequential_fused_fp32_us": seq32, "speedup_vs_sequential_fused_fp32": seq32 / p50,
            "roofline": {"bound": "hbm", "achieved": alg / (p50 * 1e-6) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (p50 * 1e-6) / 1e9 / hbm, "algorithmic_bytes": alg},
            "plan": plan,
            "one_launch": {"p50_us": p50_1, "p99_us": float(np.percentile(t1, 99)),
                           "instance_frames_per_s": 64 * 1e6 / p50_1, "autotune": tuned1, "plan": plan1,
                           "what": "the whole batch in one persistent launch per frame (the autotuner bounded to "
                                   "one launch); p50_us above is the autotuner's free choice of launches"}}


def bench_batch_sharded(torch, fewha, dev, flush, n_frames, dist, rank, world):
    """The 64 uneven instances partitioned over the ranks (no collective in
    the solve: each rank its own batch's fused launch per frame);
    the slowest rank's p50 sets the job's batch-frame time."""
    from paper_2009_00946_b300 import shard
    cfgs = configs.c4_batch(64)
    sb = shard.ShardedBatch(cfgs, rank, world, k_rr=K_RR)
    t = [0.0]
    if sb.batch is not None:
        B = sb.batch
        per = [synth.random_slopes(c, 7).astype(np.float32) for c in B.cfgs]
        s = torch.from_numpy(B.concat_slopes(per)).to(dev)
        lay = torch.empty(B.N, dtype=torch.float32, device=dev)
        st = B.stream
        for _ in range(5):
            B.frame(s, N_ITER, True, lay)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_frames)]
        for k in range(n_frames):
            with torch.cuda.stream(st):
                flush.fill_(float(k & 7))
            ev[k][0].record(st)
            B.frame(s, N_ITER, True, lay)
            ev[k][1].record(st)
        st.synchronize()
        B.sync()
        t = [a.elapsed_time(b) * 1e3 for a, b in ev]
    else:
        lay = torch.zeros(0, device=dev)
    p50 = float(np.percentile(t, 50))
    got = sb.gather_layers(lay, dist, dst=0, device=dev)   # untimed: the results to rank 0
    p50_max = max_over_ranks([p50], dist, dev)[0]
    sb.close()
    out = {"workload": "64 independent instances partitioned over %d ranks (cost-balanced, no collective in the "
                       "solve), 4 warm-started iterations each, FP32, one fused launch per rank per frame" % world,
           "p50_us_slowest_rank": p50_max, "instance_frames_per_s_total": 64 * 1e6 / p50_max,
           "instances_per_rank": [len(p) for p in sb.parts], "frames": n_frames, "scaling": "strong"}
    if got is not None:
        out["gathered_instances"] = sum(1 for a in got if a is not None and np.isfinite(a).all())
    return out


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (replicas: the slowest rank
    sets the job's latency); identity without a process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu().tolist()]


def phase_breakdown(S, pool_dev, n_iter=N_ITER, dump=None):
    """One traced non-replacement frame: critical-path time of each phase (the
    latest CTA's work between two barriers) and the barrier latencies (us)."""
    S.set_trace(True)
    S.set_residual_replacement(0)
    S.set_frame(pool_dev[0])
    S.solve(n_iter, warm=True)
    tr = S.trace().astype(np.int64)
    fine = S.fine_trace()
    S.set_trace(False)
    if dump:
        np.save(dump + "_barriers.npy", tr)
        np.save(dump + "_fine.npy", np.array([(c, t, v) for c, r in enumerate(fine) for t, v in r], np.int64))
    # sub-phase steps: mean over CTAs and phases of the time between marks
    names = {(10, 11): "layer_stage_rows_us", (11, 12): "layer_PT_us", (12, 13): "layer_fwd_dwt_us",
             (13, 14): "layer_update_us", (14, 15): "layer_inv_dwt_us", (13, 17): "layer_scalars_us",
             (17, 18): "layer_update_loop_us", (18, 14): "layer_update_reduce_us",
             (13, 40): "scal_enter_us", (40, 41): "scal_partials_us", (41, 42): "scal_butterfly_us",
             (42, 43): "scal_fp64_us", (43, 17): "scal_exit_us", (15, 16): "layer_store_sync_us",
             (14, 16): "layer_no_inverse_us", (20, 21): "sensor_stage_windows_us", (21, 22): "sensor_P_us",
             (22, 23): "sensor_slopes_us", (23, 24): "sensor_gammaT_store_us",
             (12, 50): "casc_cols_fwd_us", (50, 51): "casc_sync1_us", (51, 13): "casc_rows_fwd_us",
             (14, 53): "casc_rows_inv_us", (53, 54): "casc_sync2_us", (54, 15): "casc_cols_inv_us"}
    steps = {}
    for row in fine:
        for (ta, a), (tb, b) in zip(row[:-1], row[1:]):
            if (ta, tb) in names:
                steps.setdefault(names[(ta, tb)], []).append((b - a) / 1e3)
    S.set_residual_replacement(K_RR)
    work, bars = [], []
    for b in range(1, tr.shape[0]):
        work.append(float((tr[b, :, 0] - tr[b - 1, :, 1]).max()) / 1e3)
        if b < tr.shape[0] - 1:
            bars.append(float(tr[b, :, 1].max() - tr[b, :, 0].max()) / 1e3)
    sensor, layer = work[2::2], work[3::2]
    return {"rhs_sensor_us": work[0], "rhs_layer_us": work[1],
            "sensor_phase_us": float(np.mean(sensor)) if sensor else None,
            "layer_phase_us": float(np.mean(layer)) if layer else None,
            "grid_barrier_us": float(np.mean(bars)) if bars else None,
            "kernel_us": float(tr[-1, :, 0].max() - tr[0, :, 1].min()) / 1e3,
            "n_barriers": len(bars),
            "steps_mean_us": {k: float(np.mean(v)) for k, v in sorted(steps.items())},
            "steps_max_us": {k: float(np.max(v)) for k, v in sorted(steps.items())}}


def sweep_mode(args):
    """Operator and frame timings against the problem size (the paper's
    operator figures and its scaling to 300x300 subapertures), one JSON line
    per point; CUDA events on the handle's stream, warm L2."""
    from paper_2009_00946_b300 import fewha

    def lines(cfg, tag, ops, precs=(fewha.FP32, fewha.FP64)):
        for prec in precs:
            with fewha.Solver(cfg, precision=prec) as S:
                for op, name in ops:
                    us = S.time_operator(op, 50)
                    print(json.dumps({"sweep": tag, "op": name, "precision": "fp64" if prec else "fp32",
                                      "us": us, "N": S.N, "S": S.S}), flush=True)

    base = configs.c2_elt()
    for n in (64, 128, 256, 512, 1024):   # W, W^T against the layer side (one layer)
        cfg = dict(base, layers=[{"height": 0.0, "cn2": 1.0, "n": n, "levels": int(math.log2(n)) - 3}],
                   wfs=base["wfs"][:1])
        lines(cfg, "n_lay=%d" % n, [(fewha.OP_W, "W"), (fewha.OP_WT, "WT")])
    for ns in (16, 32, 64, 84, 128, 200, 300):   # P, P^T, Gamma, Gamma^T against n_s at n_lay = 128
        cfg = dict(base, wfs=[dict(w, n_sub=ns) for w in base["wfs"]])
        lines(cfg, "n_s=%d" % ns, [(fewha.OP_P, "P"), (fewha.OP_PT, "PT"), (fewha.OP_GAMMA, "Gamma"),
                                   (fewha.OP_GAMMA_T, "GammaT")])
    import torch
    for ns in (84, 128, 200, 256, 300):   # whole solve (4 iterations) against n_s, n_lay = next power of two
        nl = 1 << int(math.ceil(math.log2(ns + 1)))
        cfg = dict(base, wfs=[dict(w, n_sub=ns) for w in base["wfs"]],
                   layers=[dict(l, n=nl, levels=int(math.log2(nl)) - 3) for l in base["layers"]])
        for prec in (fewha.FP32, fewha.FP64):
            S = fewha.Solver(cfg, precision=prec, k_rr=K_RR)
            S.set_frame(np.asarray(synth.random_slopes(cfg, 3), dtype=S.np_dtype))
            for _ in range(3):
                S.solve(N_ITER, warm=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(S.stream)
            for _ in range(20):
                S.solve(N_ITER, warm=True)
            e1.record(S.stream)
            S.sync()
            print(json.dumps({"sweep": "frame n_s=%d n_lay=%d" % (ns, nl), "precision": "fp64" if prec else "fp32",
                              "path": S.describe().split(",")[1].strip(), "us": e0.elapsed_time(e1) * 1e3 / 20,
                              "N": S.N, "S": S.S}), flush=True)
            S.close()


def profile_mode(args):
    """Stream launches only (no CUDA graph), for ncu: W + K frames of
    set_frame (device) + solve + layers on the fused path."""
    import torch
    from paper_2009_00946_b300 import fewha
    cfg = workload_config()
    pool = slope_pool(cfg, args.pool)
    dev = torch.device("cuda", 0)
    pool_dev = torch.from_numpy(pool).to(dev)
    S = fewha.Solver(cfg, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR)
    out = torch.empty(S.N, dtype=torch.float32, device=dev)
    for k in range(args.warmup + args.steps):
        S.set_frame(pool_dev[k % len(pool)])
        S.solve(N_ITER, warm=True)
        S.layers(out)
    S.sync()
    print(json.dumps({"profile_mode": True, "frames": args.warmup + args.steps, "plan": S.describe(),
                      "phases": phase_breakdown(S, pool_dev, dump=args.trace_out)}), flush=True)
    S.close()


def profile_batch_mode(args):
    """Stream launches of the 64-instance batch (for ncu) in the grouping the
    autotuner chooses on this workload: the 25 instances with 256^2 layers on
    clusters of 8 with sensor tiles of at most 48 nodes per side, the other
    39 on clusters of 2 with tiles of at most 64.  W + K frames on device
    buffers, each the two launches in that order."""
    import torch
    from paper_2009_00946_b300 import fewha
    cfgs = configs.c4_batch(64)
    side = [max(l["n"] for l in c["layers"]) for c in cfgs]
    groups = [([c for c, n in zip(cfgs, side) if n == 256], 8, 48), ([c for c, n in zip(cfgs, side) if n < 256], 2, 64)]
    runs = []
    for cs, C, tile in groups:
        B = fewha.Batch(cs, k_rr=K_RR, cluster_size=C, max_tile_side=tile)
        per = [synth.random_slopes(c, 7).astype(np.float32) for c in cs]
        s = torch.from_numpy(B.concat_slopes(per)).cuda()
        lay = torch.empty(B.N, dtype=torch.float32, device="cuda")
        runs.append((B, s, lay))
    for _ in range(args.warmup + args.steps):
        for B, s, lay in runs:
            B.frame(s, N_ITER, True, lay)
    for B, _, _ in runs:
        B.sync()
    print(json.dumps({"profile_batch": True, "frames": args.warmup + args.steps,
                      "plans": [B.describe() for B, _, _ in runs]}), flush=True)
    for B, _, _ in runs:
        B.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fewha", choices=["fewha", "reference"])
    ap.add_argument("--pool", type=int, default=64, help="distinct synthetic frames, cycled")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 35-layer fit and 64-instance batch lines")
    ap.add_argument("--profile", action="store_true", help="stream launches only (for ncu), no timing")
    ap.add_argument("--profile-batch", action="store_true", help="batch launches only (for ncu), no timing")
    ap.add_argument("--sweep", action="store_true", help="operator and frame timings against the size")
    ap.add_argument("--trace-out", default=None, help="with --profile: save the raw phase traces (.npy)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile:
        profile_mode(args)
        return
    if args.profile_batch:
        profile_batch_mode(args)
        return
    if args.sweep:
        sweep_mode(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = workload_config()
    pool = slope_pool(cfg, args.pool, seed=cfg["seed"] + 100 * rank)

    # CPU oracle baseline first (rank 0, N = 1), before any CUDA call
    cpu = None
    oracle_layers = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle_layers = []
        t = cpu_oracle_latency(cfg, 30, pool, oracle_layers)[2:]
        cpu = {"value": float(np.percentile(t, 50)), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "28 ELT frames (after 2 warm-up frames), FP64 numpy oracle, one host thread (%d cores "
                         "on the host)" % os.cpu_count()}
        cpu_all = cpu_oracle_all_cores(cfg)

    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2009_00946_b300 import fewha

    dev = torch.device("cuda", local_rank)
    pool_dev = torch.from_numpy(pool).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    S = fewha.Solver(cfg, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR)
    layers_dev = torch.empty(S.N, dtype=torch.float32, device=dev)
    W, K = args.warmup, args.steps
    time_frames(S, torch, pool_dev, 0, W, layers_dev, flush)
    S.sync()

    # ---- timed region: K frames, device-resident inputs ----
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = S.launch_count()
    with ClockSampler(local_rank) as clk:
        lat = time_frames(S, torch, pool_dev, W, K, layers_dev, flush)
        S.sync()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = S.launch_count() - l0
    p50, p99 = float(np.percentile(lat, 50)), float(np.percentile(lat, 99))
    mean = float(np.mean(lat))

    # ---- kernel-level: solve duration (roofline) and per-iteration cost ----
    t4 = time_solve(S, torch, N_ITER, 100, flush)
    t100 = time_solve(S, torch, 100, 20, flush)
    per_iter = (t100 - t4) / 96.0
    phases = phase_breakdown(S, pool_dev)
    plan = S.describe()
    hbm, peak_kind = measured_peaks()

    # ---- end to end: pinned host slopes in, layers out, through fewha_frame ----
    pin_s = torch.empty(S.S, dtype=torch.float32).pin_memory()
    pin_l = torch.empty(S.N, dtype=torch.float32).pin_memory()
    host_s, host_l = pin_s.numpy(), pin_l.numpy()   # the caller's arrays, made once
    run_frame = S.bind_frame(host_s, N_ITER, warm=True, layers_out=host_l)   # the real-time loop's call
    e2e, e2e_ft, e2e_unbound = [], [], []
    n_e2e = min(K, 300)
    # warm-up of the host path (pinned mappings, both frame kinds) for two
    # seconds: host frames run slower for about a second after an nvidia-smi
    # sampler (the timed region's clock record) has exited
    t_w = time.perf_counter()
    k = 0
    while k < 50 or time.perf_counter() - t_w < 2.0:
        host_s[:] = pool[k % len(pool)]
        run_frame()
        k += 1
    for k in range(n_e2e + 5):
        host_s[:] = pool[(W + K + k) % len(pool)]
        with torch.cuda.stream(S.stream):
            flush.fill_(2.0)
        S.stream.synchronize()
        t0 = time.perf_counter()
        run_frame()
        t3 = time.perf_counter()
        e2e.append((t3 - t0) * 1e6)
        e2e_ft.append(S.frame_timing())
    # armed frames: the kernel launched (and its set-up done) before the slopes
    # are written, then fired; timed from the go to the layers in host memory
    e2e_armed = []
    for k in range(min(n_e2e, 200) + 5):
        with torch.cuda.stream(S.stream):
            flush.fill_(2.0)
        S.stream.synchronize()
        S.arm_frame(host_s, N_ITER, warm=True, layers_out=host_l, wait_s=1.0)
        host_s[:] = pool[(W + K + k) % len(pool)]   # the slopes arrive
        t0 = time.perf_counter()
        S.fire_frame()
        e2e_armed.append((time.perf_counter() - t0) * 1e6)
    e2e_armed = e2e_armed[5:]
    # the same frames through the unbound call (arguments checked every frame)
    for k in range(min(n_e2e, 100) + 5):
        host_s[:] = pool[(W + K + k) % len(pool)]
        with torch.cuda.stream(S.stream):
            flush.fill_(2.0)
        S.stream.synchronize()
        t0 = time.perf_counter()
        S.frame(host_s, N_ITER, warm=True, layers_out=host_l)
        e2e_unbound.append((time.perf_counter() - t0) * 1e6)
    e2e, e2e_ft, e2e_unbound = e2e[5:], e2e_ft[5:], e2e_unbound[5:]
    # device time of host frames, bracketed by CUDA events on the handle's
    # stream (the GPU kept busy by the flush so the host's side does not show
    # as idle time): the frame as run (the kernel launched first, the slopes
    # by the copy engine on a second stream); the graph form with the slopes
    # copied ahead of the kernel; the graph form with the slopes read by the
    # kernel through the pinned mapping, with and without the layers written
    # back through it
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]

    def dev_p50(fn):
        for k in range(50):
            with torch.cuda.stream(S.stream):
                flush.fill_(3.0)
            ev[k][0].record(S.stream)
            fn()
            ev[k][1].record(S.stream)
        S.stream.synchronize()
        return float(np.percentile([a.elapsed_time(b) * 1e3 for a, b in ev], 50))

    e2e_dev = dev_p50(run_frame)
    run_in = S.bind_frame(host_s, N_ITER, warm=True)   # slopes in, layers left on the device
    e2e_dev_in = dev_p50(run_in)
    S.set_host_transfer(False)
    e2e_dev_in_mapped = dev_p50(run_in)
    e2e_dev_mapped = dev_p50(run_frame)
    S.set_host_transfer(True)
    with ClockSampler(local_rank) as clk_l2:
        l2 = fewha.measure_l2()
    l2["clocks"] = clk_l2.summary()
    roofline = roofline_block(cfg, t4, per_iter, l2, hbm, peak_kind, fused_traffic())
    e2e_breakdown = {
        "host_prep_us": float(np.median([f["prep_us"] for f in e2e_ft])),
        "host_launch_us": float(np.median([f["launch_us"] for f in e2e_ft])),
        "host_wait_us": float(np.median([f["wait_us"] for f in e2e_ft])),
        "library_call_us": float(np.median([f["total_us"] for f in e2e_ft])),
        "python_call_us": float(np.median([e - f["total_us"] for e, f in zip(e2e, e2e_ft)])),
        "unbound_call_p50_us": float(np.percentile(e2e_unbound, 50)),
        "armed_frame_p50_us": float(np.percentile(e2e_armed, 50)),
        "armed_frame_p99_us": float(np.percentile(e2e_armed, 99)),
        "library_call_p99_us": float(np.percentile([f["total_us"] for f in e2e_ft], 99)),
        "host_wait_p99_us": float(np.percentile([f["wait_us"] for f in e2e_ft], 99)),
        "device_frame_with_host_io_us": e2e_dev,
        "host_io_in_kernel_us": e2e_dev - p50,
        "slopes_copy_ahead_of_kernel_us": e2e_dev_in - p50,
        "slopes_in_through_mapping_us": e2e_dev_in_mapped - p50,
        "layers_write_in_kernel_us": e2e_dev_mapped - e2e_dev_in_mapped,
        "host_io_bytes": (S.S + S.N) * 4,
        "host_io_gbs": (S.S + S.N) * 4 / max(e2e_dev - p50, 1e-3) / 1e3,
        "what": "library_call = prep + launch + wait (host steady clock inside fewha_frame); python_call = "
                "the e2e time of a frame minus its library_call (the bound call's interpreter and ctypes share); "
                "unbound_call = the same frames through Solver.frame, whose arguments are checked every frame; armed_frame = "
                "fewha_frame_arm before the slopes are written (the launch and the kernel's set-up happen then), "
                "timed from fewha_frame_fire to the layers in host memory; host_io_in_kernel = device time of a host frame "
                "(as run: the kernel launched first, the slopes by the copy engine on a second stream while it sets up) "
                "minus the device p50; slopes_copy_ahead_of_kernel = the graph form with the slopes' copy before the "
                "kernel, slopes_in_through_mapping = the kernel reading them through the pinned mapping (layers left on "
                "the device in both), layers_write_in_kernel = the layers written through the mapping (mapped form with "
                "and without them)"}

    # ---- the plain FP64 path (one kernel per operator) on the same frames ----
    P64 = fewha.Solver(cfg, precision=fewha.FP64, k_rr=K_RR)
    pool64 = pool_dev.double()
    lay64 = torch.empty(P64.N, dtype=torch.float64, device=dev)
    n64 = min(K, 200)
    time_frames(P64, torch, pool64, 0, 5, lay64, flush)
    lat64 = time_frames(P64, torch, pool64, 5, n64, lay64, flush)
    p64_t4 = time_solve(P64, torch, N_ITER, 10, flush)
    p64_t20 = time_solve(P64, torch, 20, 5, flush)
    p64_iter = (p64_t20 - p64_t4) / 16.0
    P64.close()

    parity = parity_vs_oracle(fewha, cfg, pool, oracle_layers) if oracle_layers else None

    # ---- the other workloads: 35-layer frame with the mirror fit, 64-instance batch ----
    extra = {}
    if not args.no_extra:
        extra["elt_dm_frame"] = bench_elt_dm_frame(torch, fewha, dev, flush, min(K, 200))
        extra["maory_frame"] = bench_maory_frame(torch, fewha, dev, flush, min(K, 200))
        extra["ltao_frame"] = bench_mode_frame(torch, fewha, dev, flush, min(K, 200), "ltao")
        extra["moao_frame"] = bench_mode_frame(torch, fewha, dev, flush, min(K, 200), "moao")
        extra["autograd_batch32"] = bench_autograd(torch, fewha, dev, flush)
        if world > 1:
            extra["batch64_sharded"] = bench_batch_sharded(torch, fewha, dev, flush, min(K, 30), dist, rank, world)
        else:
            extra["batch64"] = bench_batch(torch, fewha, dev, flush, min(K, 30))

    # max over ranks
    p50, p99, mean, per_iter = max_over_ranks([p50, p99, mean, per_iter], dist, dev)
    if rank != 0:
        S.close()
        if dist:
            dist.destroy_process_group()
        return
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": p50, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": mean / 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (FP64 dots/scalars)", "data": "synthetic",
        "config": config_block(cfg, {"path": "fused persistent kernel, CUDA graph per frame",
                                     "parallelism": "replicas" if world > 1 else "1 GPU"}),
        "p50_us": p50, "p99_us": p99,
        "pcg_iter_per_s": 1e6 / per_iter if per_iter > 0 else None,
        "us_per_pcg_iter": per_iter,
        "frames_per_s_total": world * 1e6 / mean,
        "plain_fp64": {"p50_us": float(np.percentile(lat64, 50)), "p99_us": float(np.percentile(lat64, 99)),
                       "us_per_pcg_iter": p64_iter, "pcg_iter_per_s": 1e6 / p64_iter if p64_iter > 0 else None,
                       "frames": n64},
        "e2e": {"value": float(np.percentile(e2e, 50)), "unit": UNIT, "p99": float(np.percentile(e2e, 99)),
                "h2d_bytes_per_step": S.S * 4, "d2h_bytes_per_step": S.N * 4, "frames": n_e2e,
                "breakdown": e2e_breakdown,
                "how": "fewha_frame through Solver.bind_frame (the buffers bound once, the slopes refilled in place each frame) with pinned host slopes and layers: the kernel launched first, the slopes brought in by the copy engine on a second stream while it does its set-up, the layers written by the kernel through their device mapping, the host waiting on the mapped completion word; host wall clock per frame"},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "l2_measured": l2,
        "clocks": clocks,
        "phases": phases,
        **extra,
        "plan": plan,
    }
    if cpu:
        line["cpu_baseline"] = cpu
        line["cpu_baseline_all_cores"] = cpu_all
    if parity:
        line["parity"] = parity
    print(json.dumps(line), flush=True)
    S.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
