"""Long-run parity of the fused FP32 frame path with the FP64 oracle.

The warm restart of Alg. 1 carries the residual r and the coefficients c from
frame to frame, so FP32 rounding could drift over many frames; the residual
replacement every k_rr frames (r = b - M c) is what bounds it.  This helper
runs the ELT bulk workload (6 LGS 84x84, 9 layers 128^2, 4 warm-started PCG
iterations per frame, replacement every 10 frames) for many consecutive
frozen-flow frames through the library and through the oracle, and compares
the layers of every frame.

Pipeline (all CPU work in processes started with `spawn` before any CUDA
call): worker processes manufacture the slopes of disjoint frame ranges; one
process runs the oracle over the frames in order (each frame depends on the
previous one) and sends the layers of every frame back; the main process runs
the same slopes, rounded to FP32 (both sides see identical inputs), through
fewha_frame and compares frame by frame.

    python tests/long_run.py --frames 1000 [--out result.json]
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ITER = 4
K_RR = 10


def _slopes_chunk(args):
    cfg, start, count = args
    from paper_2009_00946_b300 import synth
    atm = synth.Atmosphere(cfg)
    return start, np.stack([atm.slopes(start + k) for k in range(count)]).astype(np.float32)


def _oracle_run(cfg, path, n_frames, q):
    from oracle import fewha_oracle as fo
    S = np.load(path, mmap_mode="r")
    R = fo.Reconstructor(cfg)
    for k in range(n_frames):
        R.frame(np.asarray(S[k], dtype=np.float64), N_ITER, warm=True, k_rr=K_RR)
        q.put((k, R.layers()))


def run(n_frames: int, workers: int | None = None, cfg=None, form: int = -1) -> dict:
    import multiprocessing as mp

    from paper_2009_00946_b300 import configs
    cfg = cfg or configs.c2_elt()
    ctx = mp.get_context("spawn")
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 2))
    t0 = time.time()
    chunk = max(1, -(-n_frames // workers))
    jobs = [(cfg, s, min(chunk, n_frames - s)) for s in range(0, n_frames, chunk)]
    tmp = tempfile.mkdtemp(prefix="fewha_long_")
    path = os.path.join(tmp, "slopes.npy")
    with ctx.Pool(len(jobs)) as pool:
        parts = dict(pool.map(_slopes_chunk, jobs))
    slopes = np.concatenate([parts[s] for _, s, _ in jobs])
    np.save(path, slopes)
    t_slopes = time.time() - t0
    q = ctx.Queue(maxsize=64)
    orc = ctx.Process(target=_oracle_run, args=(cfg, path, n_frames, q), daemon=True)
    orc.start()

    import torch  # noqa: F401  (CUDA from here on)
    from paper_2009_00946_b300 import fewha
    sides = [l["n"] for l in cfg["layers"]]
    S = fewha.Solver(cfg, precision=fewha.FP32, path=fewha.PATH_FUSED, k_rr=K_RR)
    if form >= 0:
        S.set_layer_transform(form)
    plan = S.describe()
    out = np.empty(S.N, np.float32)
    rel, emax, border = [], [], []
    try:
        for k in range(n_frames):
            S.frame(slopes[k], N_ITER, warm=True, layers_out=out)
            kk, ref = q.get(timeout=600)
            assert kk == k
            got = out.astype(np.float64)
            rel.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
            o, e, b = 0, 0.0, 0.0
            for n in sides:
                d = np.abs(got[o:o + n * n] - ref[o:o + n * n]).reshape(n, n)
                sc = float(np.max(np.abs(ref[o:o + n * n])))
                e = max(e, float(d.max()) / sc)
                b = max(b, max(float(d[:2].max()), float(d[-2:].max()), float(d[:, :2].max()),
                               float(d[:, -2:].max())) / sc)
                o += n * n
            emax.append(e)
            border.append(b)
    finally:
        S.close()
        orc.join(timeout=60)
        try:
            os.remove(path)
            os.rmdir(tmp)
        except OSError:
            pass
    r = np.asarray(rel)
    repl = [k for k in range(n_frames) if K_RR and k > 0 and k % K_RR == 0]
    return {"frames": n_frames, "workload": cfg["name"], "n_iter": N_ITER, "k_rr": K_RR,
            "layers_rel_l2_max": float(r.max()), "layers_rel_l2_median": float(np.median(r)),
            "layers_rel_l2_p99": float(np.percentile(r, 99)), "worst_frame": int(r.argmax()),
            "layers_rel_l2_last_50_mean": float(r[-50:].mean()), "layers_rel_l2_first_50_mean": float(r[:50].mean()),
            "elementwise_max_over_grid_max": float(max(emax)), "border_max_over_grid_max": float(max(border)),
            "replacement_frames": len(repl), "tolerance": 1e-4,
            "slopes_workers": len(jobs), "slopes_s": t_slopes, "total_s": time.time() - t0, "plan": plan,
            "per_frame_rel_l2": [float(x) for x in r]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=1000)
    ap.add_argument("--workers", type=int, default=None)
    ap.add_argument("--out", default=None)
    ap.add_argument("--form", type=int, default=-1, help="fused layer transform (-1 automatic, 0, 1)")
    a = ap.parse_args()
    res = run(a.frames, a.workers, form=a.form)
    short = {k: v for k, v in res.items() if k != "per_frame_rel_l2"}
    print(json.dumps(short), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)
    return 0 if res["layers_rel_l2_max"] < 1e-4 else 1


if __name__ == "__main__":
    sys.exit(main())
