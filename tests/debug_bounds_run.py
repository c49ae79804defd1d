"""The library's debug build (bounds checks at every gather and scatter) on the
GPU, against the FP64 oracle.

Run with FEWHA_DEBUG=1 in the environment, so that the binding loads
libfewha_debug.so: every case below drives one part of the hot path through
the C ABI -- the fused frame kernel with both layer transforms, ragged tiles,
the LGS tip-tilt filter and the mirror fit; pinned host frames (armed and
fired at once) and an explicitly armed frame; the plain operator kernels in
FP64 and FP32; the batched launch, one and two launches per frame; the taped
solve and its reverse mode; the no-allocation transform -- compares its results with the oracle and reads the
violations the checks recorded (fewha_debug_bounds).  A check that fails
skips its access, so a violation shows here as a count (and usually as a
parity error), never as a memory fault.

    FEWHA_DEBUG=1 python tests/debug_bounds_run.py [--out result.json]

Prints one JSON object: {"debug_build": bool, "cases": {name: {"count",
"site", "index", "err", "tol"}}}.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


class Violation(RuntimeError):
    pass


_SEEN = {"count": 0, "site": None, "index": None}


def _stop_on_violation(fw):
    """Reads the records after a step; the first violation ends the run (a
    skipped access leaves a buffer unwritten, so nothing after it is run)."""
    d = fw.debug_bounds()
    if d["count"]:
        _SEEN.update(count=_SEEN["count"] + d["count"], site=_SEEN["site"] or d["site"],
                     index=_SEEN["index"] if _SEEN["site"] else d["index"])
        raise Violation("%d violations, first at %s index %s" % (d["count"], d["site"], d["index"]))


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_frames(cfg, n_frames, fit=False):
    from oracle import fewha_oracle as fo
    from paper_2009_00946_b300 import synth
    S_in, _ = synth.frames(cfg, n_frames)
    R = fo.Reconstructor(cfg)
    ref = []
    for k in range(n_frames):
        if fit:
            o = R.frame(S_in[k], 4, warm=True, k_rr=10, gain=0.5, n_fit=8)
            ref.append((R.layers(), o["a"].copy()))
        else:
            R.frame(S_in[k], 4, warm=True, k_rr=10)
            ref.append((R.layers(), None))
    return S_in, ref


def case_frames(fw, cfg, n_frames, precision, path, form=None, fit=False):
    """Host frames through fewha_frame; the worst relative error over the
    frames (layers, and mirror commands with the fit)."""
    S_in, ref = _oracle_frames(cfg, n_frames, fit)
    dt = np.float64 if precision == fw.FP64 else np.float32
    worst = 0.0
    with fw.Solver(cfg, precision=precision, path=path, k_rr=10) as S:
        if form is not None:
            S.set_layer_transform(form)
        for k in range(n_frames):
            lay = np.empty(S.N, dt)
            a = np.empty(S.NA, dt) if fit else None
            S.frame(np.ascontiguousarray(S_in[k], dtype=dt), 4, warm=True, gain=0.5, n_fit=8, layers_out=lay,
                    dm_out=a)
            _stop_on_violation(fw)
            worst = max(worst, rel(lay, ref[k][0]))
            if fit:
                worst = max(worst, rel(a, ref[k][1]))
    return worst


def case_batch(fw, n_frames=3):
    from paper_2009_00946_b300 import configs
    cfgs = [configs.c4_instance(i) for i in (1, 6, 24, 56)]
    refs = [_oracle_frames(c, n_frames) for c in cfgs]
    worst = 0.0
    with fw.Batch(cfgs, k_rr=10) as B:
        out = np.empty(B.N, np.float32)
        for k in range(n_frames):
            B.frame(B.concat_slopes([r[0][k].astype(np.float32) for r in refs]), 4, warm=True, layers_out=out)
            _stop_on_violation(fw)
            for i, lay in enumerate(B.split_layers(out)):
                worst = max(worst, rel(lay, refs[i][1][k][0]))
    return worst


def case_frames_pinned(fw, torch, cfg, n_frames):
    """Host frames on pinned buffers (run as armed frames fired at once: the
    kernel launched first, the slopes copied in on a second stream) and one
    explicitly armed frame; the worst relative error of the layers."""
    S_in, ref = _oracle_frames(cfg, n_frames)
    worst = 0.0
    with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_FUSED, k_rr=10) as S:
        ps = torch.empty(S.S, dtype=torch.float32).pin_memory()
        pl = torch.empty(S.N, dtype=torch.float32).pin_memory()
        for k in range(n_frames):
            if k == n_frames - 1:
                S.arm_frame(ps.numpy(), 4, warm=True, layers_out=pl.numpy(), wait_s=5.0)
                ps.numpy()[:] = S_in[k]
                S.fire_frame()
            else:
                ps.numpy()[:] = S_in[k]
                S.frame(ps.numpy(), 4, warm=True, layers_out=pl.numpy())
            _stop_on_violation(fw)
            worst = max(worst, rel(pl.numpy(), ref[k][0]))
    return worst


def case_batch_grouped(fw, n_frames=3):
    """A batch split by hand into two launches (the 256^2 instances apart)."""
    from paper_2009_00946_b300 import configs
    cfgs = [configs.c4_instance(i) for i in (1, 6, 7, 24, 8)]
    refs = [_oracle_frames(c, n_frames) for c in cfgs]
    group = [0 if max(l["n"] for l in c["layers"]) == 256 else 1 for c in cfgs]
    worst = 0.0
    with fw.Batch(cfgs, k_rr=10, max_tile_side=48) as B:
        B.set_groups(group)
        out = np.empty(B.N, np.float32)
        for k in range(n_frames):
            B.frame(B.concat_slopes([r[0][k].astype(np.float32) for r in refs]), 4, warm=True, layers_out=out)
            _stop_on_violation(fw)
            for i, lay in enumerate(B.split_layers(out)):
                worst = max(worst, rel(lay, refs[i][1][k][0]))
    return worst


def case_operators(fw):
    """M applied by the plain FP64 kernels (P, Gamma, C^-1, Gamma^T, P^T, the
    DWTs and alpha D) against the oracle."""
    from oracle import fewha_oracle as fo
    from paper_2009_00946_b300 import synth
    from _cases import ragged_cfg
    cfg = ragged_cfg()
    g = fo.Geometry(cfg)
    with fw.Solver(cfg, precision=fw.FP64) as S:
        x = synth.random_coeffs(cfg, 7)
        return rel(S.apply_M(x), fo.apply_M(g, x))


def case_autograd(fw, torch):
    """Taped FP64 solve and its reverse mode on the autograd configuration:
    the loss gradients against the oracle's adjoint."""
    from oracle import fewha_oracle as fo
    from paper_2009_00946_b300 import configs, synth
    cfg = configs.c5_autograd()
    g = fo.Geometry(cfg)
    pr = g.default_params()
    Jinv = 1.0 / fo.jacobi_diag(g, pr)
    S, T = synth.frames(cfg, 1)
    with fw.Solver(cfg, precision=fw.FP64) as S_:
        with torch.cuda.stream(S_.stream):
            sd = torch.from_numpy(np.asarray(S[0])).to("cuda", torch.float64)
            tape = torch.empty(S_.tape_bytes(4), dtype=torch.uint8, device="cuda")
            phi = torch.empty(S_.N, dtype=torch.float64, device="cuda")
            S_.solve_taped(sd, 4, tape, phi)
            phibar = 2.0 * (phi - torch.from_numpy(T[0]).to("cuda", torch.float64))
            gg = torch.empty(S_.n_layers, dtype=torch.float64, device="cuda")
            ga = torch.empty(1, dtype=torch.float64, device="cuda")
            gw = torch.empty(S_.n_wfs, dtype=torch.float64, device="cuda")
            gs = torch.empty_like(sd)
            S_.backward(sd, 4, tape, phibar, gg, ga, gw, gs)
        S_.sync()
    _, ogg, oga, ogw, ogs = fo.solve_loss_grad(g, pr, Jinv, S[0], T[0], 4, with_slopes=True)
    return max(rel(gg.cpu().numpy(), ogg), abs(float(ga.cpu()) - oga) / abs(oga), rel(gw.cpu().numpy(), ogw),
               rel(gs.cpu().numpy(), ogs))


def case_noalloc(fw, torch):
    """fewha_layers_noalloc on a stack of mixed sides and level counts against
    the oracle's synthesis."""
    from oracle import fewha_oracle as fo
    from paper_2009_00946_b300 import configs, synth
    cfg = configs.c1_plain()
    base = cfg["layers"][0]
    cfg["layers"] = [dict(base, height=0.0, n=64, levels=2), dict(base, height=3000.0, n=128, levels=4),
                     dict(base, height=6000.0, n=256, levels=5), dict(base, height=9000.0, n=32, levels=3)]
    c = synth.random_coeffs(cfg, 300).astype(np.float32)
    want, o = [], 0
    for l in cfg["layers"]:
        n = l["n"]
        want.append(fo.inv_dwt2(c[o:o + n * n].astype(np.float64).reshape(n, n), l["levels"]).ravel())
        o += n * n
    L = len(cfg["layers"])
    ns = (ctypes.c_int * L)(*[l["n"] for l in cfg["layers"]])
    Js = (ctypes.c_int * L)(*[l["levels"] for l in cfg["layers"]])
    c_dev = torch.from_numpy(c).to("cuda")
    out = torch.empty_like(c_dev)
    torch.cuda.synchronize()
    msg = ctypes.create_string_buffer(256)
    st = fw.lib().fewha_layers_noalloc(ctypes.c_void_p(c_dev.data_ptr()), ctypes.c_void_p(out.data_ptr()), L, ns, Js,
                                       None, msg, 256)
    if st:
        raise RuntimeError(msg.value.decode())
    torch.cuda.synchronize()
    return rel(out.cpu().numpy(), np.concatenate(want))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    from paper_2009_00946_b300 import configs, fewha as fw
    from _cases import ragged_cfg
    assert torch.cuda.is_available(), "needs a GPU"
    torch.cuda.set_device(0)
    st = fw.debug_bounds()   # clears anything left from start-up
    tt = configs.mcao_small()
    tt["lgs_tip_tilt_filter"] = True
    cases = [
        ("c1_plain_fp64", 1e-10, lambda: case_frames(fw, configs.c1_plain(), 3, fw.FP64, fw.PATH_PLAIN)),
        ("ragged_plain_fp32", 1e-4, lambda: case_frames(fw, ragged_cfg(), 3, fw.FP32, fw.PATH_PLAIN)),
        ("ragged_fused_fp32", 1e-4, lambda: case_frames(fw, ragged_cfg(), 12, fw.FP32, fw.PATH_FUSED)),
        ("elt_fused_level_stacked", 1e-4, lambda: case_frames(fw, configs.c2_elt(), 12, fw.FP32, fw.PATH_FUSED, 1)),
        ("elt_fused_row_stripes", 1e-4, lambda: case_frames(fw, configs.c2_elt(), 3, fw.FP32, fw.PATH_FUSED, 0)),
        ("mcao_tt_fit_fused", 1e-4, lambda: case_frames(fw, tt, 4, fw.FP32, fw.PATH_FUSED, fit=True)),
        ("mcao_tt_fit_plain_fp64", 1e-10, lambda: case_frames(fw, tt, 2, fw.FP64, fw.PATH_PLAIN, fit=True)),
        ("moao_fit_fused", 1e-4, lambda: case_frames(fw, configs.ao_mode_small("moao"), 3, fw.FP32, fw.PATH_FUSED,
                                                     fit=True)),
        ("ltao_fit_fused", 1e-4, lambda: case_frames(fw, configs.ao_mode_small("ltao"), 3, fw.FP32, fw.PATH_FUSED,
                                                     fit=True)),
        ("batch_4_instances", 1e-4, lambda: case_batch(fw)),
        ("batch_grouped_two_launches", 1e-4, lambda: case_batch_grouped(fw)),
        ("elt_fused_pinned_host_and_armed", 1e-4, lambda: case_frames_pinned(fw, torch, configs.c2_elt(), 4)),
        ("operators_fp64", 1e-12, lambda: case_operators(fw)),
        ("autograd_fp64", 1e-8, lambda: case_autograd(fw, torch)),
        ("noalloc_mixed_levels", 1e-6, lambda: case_noalloc(fw, torch)),
    ]
    res = {"debug_build": st["debug_build"], "cases": {}}
    stop = not st["debug_build"]
    for name, tol, fn in cases:
        if stop:
            res["cases"][name] = {"tol": tol, "err": None, "exception": "not run", "count": 0}
            continue
        rec = {"tol": tol}
        _SEEN.update(count=0, site=None, index=None)
        try:
            rec["err"] = float(fn())
        except Exception as e:   # reported; a violation or an error ends the run
            rec["err"] = None
            rec["exception"] = "%s: %s" % (type(e).__name__, e)
            stop = True
        torch.cuda.synchronize()
        d = fw.debug_bounds()
        rec.update(count=_SEEN["count"] + d["count"], site=_SEEN["site"] or d["site"],
                   index=_SEEN["index"] if _SEEN["site"] else d["index"])
        stop = stop or rec["count"] > 0
        res["cases"][name] = rec
        print(name, rec, file=sys.stderr, flush=True)
    line = json.dumps(res)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")
    print(line)


if __name__ == "__main__":
    main()
