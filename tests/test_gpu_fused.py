"""Parity of the fused persistent FP32 frame kernel with the FP64 oracle (<= 1e-4
relative L2 on layers), through the C ABI, plus determinism, ragged sizes, the
bounded-barrier timeout status and the graph-captured frame."""

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

from _cases import elementwise_check, ragged_cfg

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


def _fused(fw, cfg, **kw):
    S = fw.Solver(cfg, precision=fw.FP32, **kw)
    S.set_path(fw.PATH_FUSED)        # raises if the fused path is unavailable
    return S


@pytest.fixture(scope="module")
def elt_frames():
    cfg = configs.c2_elt()
    S_in, _ = synth.frames(cfg, 13)
    R = fo.Reconstructor(cfg)
    ref = []
    for k in range(13):
        R.frame(S_in[k], 4, warm=True, k_rr=10)
        ref.append((R.layers(), R.state.c.copy()))
    return cfg, S_in.astype(np.float32), ref


def test_fused_elt_frames_match_oracle(fw, elt_frames):
    """ELT bulk, 4 warm iterations per frame, 13 frames across the residual
    replacement of frame 10: layers and coefficients <= 1e-4."""
    cfg, S_in, ref = elt_frames
    sides = [l["n"] for l in cfg["layers"]]
    with _fused(fw, cfg, k_rr=10) as S:
        for k in range(13):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            S.sync()
            assert rel(S.layers(), ref[k][0]) < 1e-4, k
            assert rel(S.vector(fw.VEC_C), ref[k][1]) < 1e-4, k
            elementwise_check(S.layers(), ref[k][0], sides, 1e-3, what=k)


def test_fused_matches_plain_fp32(fw, elt_frames):
    """The fused and the plain FP32 paths evaluate the same recurrence with
    different summation orders (the fused DWT is distributed), each within a
    few 1e-5 of the FP64 oracle, so they agree to the sum of their errors."""
    cfg, S_in, _ = elt_frames
    with _fused(fw, cfg, k_rr=10) as A, fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN, k_rr=10) as B:
        for k in range(12):
            for S in (A, B):
                S.set_frame(S_in[k])
                S.solve(4, warm=True)
                S.sync()
            assert rel(A.vector(fw.VEC_C), B.vector(fw.VEC_C).astype(np.float64)) < 5e-5, k
            assert rel(A.vector(fw.VEC_R), B.vector(fw.VEC_R).astype(np.float64)) < 1e-3, k


def test_fused_bit_deterministic(fw, elt_frames):
    cfg, S_in, _ = elt_frames
    outs = []
    for _ in range(2):
        with _fused(fw, cfg) as S:
            for k in range(3):
                S.set_frame(S_in[k])
                S.solve(4, warm=True)
            S.sync()
            outs.append((S.vector(fw.VEC_C), S.layers()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("name", ["c1_plain", "c5_autograd", "ragged"])
def test_fused_small_and_ragged_geometries(fw, name):
    cfg = ragged_cfg() if name == "ragged" else configs.ALL[name]()
    S_in, _ = synth.frames(cfg, 3)
    R = fo.Reconstructor(cfg)
    with _fused(fw, cfg, k_rr=2) as S:
        for k in range(3):
            R.frame(S_in[k], 6, warm=(k > 0), k_rr=2)
            S.set_frame(S_in[k].astype(np.float32))
            S.solve(6, warm=(k > 0))
            S.sync()
            assert rel(S.layers(), R.layers()) < 1e-4, (name, k)
            elementwise_check(S.layers(), R.layers(), [l["n"] for l in cfg["layers"]], 1e-3, what=(name, k))


def test_fused_timeout_reported_and_recoverable(fw, elt_frames):
    """Barrier budget 0: every grid barrier expires at once; the kernel runs to
    its end without waiting and the TIMEOUT status is returned.  The context
    stays usable: after restoring the state the next frame is correct."""
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg) as S:
        S.set_frame(S_in[0])
        S.solve(4, warm=True)
        S.sync()
        state = S.get_state()
        S.set_barrier_budget(0)
        S.set_frame(S_in[1])
        S.solve(4, warm=True)
        with pytest.raises(fw.FewhaError) as ei:
            S.sync()
        assert ei.value.name == "TIMEOUT"
        S.set_barrier_budget(1 << 31)
        S.set_state(*state, frame_count=1)
        S.set_frame(S_in[1])
        S.solve(4, warm=True)
        S.sync()
        assert rel(S.layers(), ref[1][0]) < 1e-4


def test_fused_nan_slopes_reported(fw):
    cfg = configs.c2_elt()
    g = fo.Geometry(cfg)
    s = synth.random_slopes(cfg, 4).astype(np.float32)
    active = int(np.flatnonzero(g.mask[2].ravel() == 1)[5])
    s[g.soff[2] + active] = np.inf
    with _fused(fw, cfg) as S:
        S.set_frame(s)
        S.solve(2, warm=False)
        with pytest.raises(fw.FewhaError) as ei:
            S.sync()
        assert ei.value.name == "INPUT"


def test_fused_graph_frame_host_and_device(fw, elt_frames):
    import torch
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as A, _fused(fw, cfg, k_rr=10) as B:
        lb = np.empty(A.N, np.float32)
        dev_s = torch.empty(A.S, dtype=torch.float32, device="cuda")
        dev_l = torch.empty(A.N, dtype=torch.float32, device="cuda")
        for k in range(12):
            pin = torch.from_numpy(S_in[k]).pin_memory()
            A.frame(pin.numpy(), 4, warm=True, layers_out=lb)
            with torch.cuda.stream(B.stream):
                dev_s.copy_(torch.from_numpy(S_in[k]).to("cuda", non_blocking=False))
            B.stream.synchronize()
            B.frame(dev_s, 4, warm=True, layers_out=dev_l)
            B.sync()
            assert rel(lb, ref[k][0]) < 1e-4, k
            assert np.array_equal(lb, dev_l.cpu().numpy()), k


def test_fused_host_frames_pinned_and_completion_word(fw, elt_frames):
    """Host frames with pinned slopes and pinned layers (the kernel reads and
    writes them through their device mapping and reports through the mapped
    completion word, no stream wait): bit-identical to device frames, the
    replacement frames included, and errors come back through the word: the
    INPUT status for non-finite slopes, TIMEOUT for expired barriers, after
    which the handle recovers."""
    import torch
    cfg, S_in, ref = elt_frames
    g = fo.Geometry(cfg)
    with _fused(fw, cfg, k_rr=10) as A, _fused(fw, cfg, k_rr=10) as B:
        pin_s = torch.empty(A.S, dtype=torch.float32).pin_memory()
        pin_l = torch.empty(A.N, dtype=torch.float32).pin_memory()
        dev_s = torch.empty(A.S, dtype=torch.float32, device="cuda")
        dev_l = torch.empty(A.N, dtype=torch.float32, device="cuda")
        for k in range(11):
            pin_s.numpy()[:] = S_in[k]
            A.frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy())
            dev_s.copy_(torch.from_numpy(S_in[k]).cuda())
            torch.cuda.synchronize()
            B.frame(dev_s, 4, warm=True, layers_out=dev_l)
            B.sync()
            assert np.array_equal(pin_l.numpy(), dev_l.cpu().numpy()), k
            assert rel(pin_l.numpy(), ref[k][0]) < 1e-4, k
        state = A.get_state()
        bad = S_in[11].copy()
        active = int(np.flatnonzero(g.mask[2].ravel() == 1)[5])
        bad[g.soff[2] + active] = np.inf
        pin_s.numpy()[:] = bad
        with pytest.raises(fw.FewhaError) as ei:
            A.frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy())
        assert ei.value.name == "INPUT"
        A.set_barrier_budget(0)
        pin_s.numpy()[:] = S_in[11]
        A.set_state(*state, frame_count=11)
        with pytest.raises(fw.FewhaError) as ei:
            A.frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy())
        assert ei.value.name == "TIMEOUT"
        A.set_barrier_budget(1 << 31)
        A.set_state(*state, frame_count=11)
        A.frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy())
        assert rel(pin_l.numpy(), ref[11][0]) < 1e-4


def test_bound_frames_and_both_host_transfers_bit_identical(fw, elt_frames):
    """Solver.bind_frame (buffers bound once, the slopes refilled in place
    each frame) and both ways host slopes reach the kernel -- one copy-engine
    transfer (the default) or the kernel's reads through the pinned mapping --
    give the device frames' layers bit for bit, across the replacement frame."""
    import torch
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as A, _fused(fw, cfg, k_rr=10) as B, _fused(fw, cfg, k_rr=10) as C:
        C.set_host_transfer(False)
        bufs = [(torch.empty(A.S, dtype=torch.float32).pin_memory(), torch.empty(A.N, dtype=torch.float32).pin_memory())
                for _ in range(2)]
        runA = A.bind_frame(bufs[0][0].numpy(), 4, warm=True, layers_out=bufs[0][1].numpy())
        runC = C.bind_frame(bufs[1][0].numpy(), 4, warm=True, layers_out=bufs[1][1].numpy())
        dev_s = torch.empty(A.S, dtype=torch.float32, device="cuda")
        dev_l = torch.empty(A.N, dtype=torch.float32, device="cuda")
        for k in range(12):
            for s_, _ in bufs:
                s_.numpy()[:] = S_in[k]
            runA()
            runC()
            dev_s.copy_(torch.from_numpy(S_in[k]).cuda())
            torch.cuda.synchronize()
            B.frame(dev_s, 4, warm=True, layers_out=dev_l)
            B.sync()
            want = dev_l.cpu().numpy()
            assert np.array_equal(bufs[0][1].numpy(), want), k
            assert np.array_equal(bufs[1][1].numpy(), want), k
            assert rel(want, ref[k][0]) < 1e-4, k


def test_host_frame_after_enqueued_device_frame(fw, elt_frames):
    """A pinned host frame (run as an armed frame fired at once, its slopes
    copied into the handle's buffer on a second stream) issued while a device
    frame of the same handle is still enqueued -- a device frame copies its
    slopes into that buffer as it runs -- gives the same layers, bit for bit,
    as the two frames run one after the other with a synchronisation between."""
    import torch
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as A, _fused(fw, cfg, k_rr=10) as B:
        ps = torch.empty(A.S, dtype=torch.float32).pin_memory()
        pl = torch.empty(A.N, dtype=torch.float32).pin_memory()
        ql = torch.empty(A.N, dtype=torch.float32).pin_memory()
        dev_s = [torch.from_numpy(S_in[k]).cuda() for k in range(6)]
        dev_l = torch.empty(A.N, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for k in range(0, 6, 2):
            A.frame(dev_s[k], 4, warm=True, layers_out=dev_l)   # enqueued only
            ps.numpy()[:] = S_in[k + 1]
            A.frame(ps.numpy(), 4, warm=True, layers_out=pl.numpy())
            B.frame(dev_s[k], 4, warm=True, layers_out=dev_l)
            B.sync()
            B.frame(ps.numpy(), 4, warm=True, layers_out=ql.numpy())
            assert np.array_equal(pl.numpy(), ql.numpy()), k
            assert rel(pl.numpy(), ref[k + 1][0]) < 1e-4, k


def test_armed_frames_bit_identical(fw, elt_frames):
    """Frames armed ahead of their slopes (fewha_frame_arm: the kernel launched
    and waiting; the slopes written afterwards; fewha_frame_fire) give the
    device frames' layers bit for bit, across the replacement frame, with the
    slopes brought in at the fire by the copy engine (default) or read by the
    kernel through the pinned mapping; while a frame is armed the handle
    refuses other work."""
    import torch
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as A, _fused(fw, cfg, k_rr=10) as B, _fused(fw, cfg, k_rr=10) as C:
        C.set_host_transfer(False)
        bufs = [(torch.empty(A.S, dtype=torch.float32).pin_memory(), torch.empty(A.N, dtype=torch.float32).pin_memory())
                for _ in range(2)]
        dev_s = torch.empty(A.S, dtype=torch.float32, device="cuda")
        dev_l = torch.empty(A.N, dtype=torch.float32, device="cuda")
        for k in range(12):
            for S_, (ps, pl) in ((A, bufs[0]), (C, bufs[1])):
                S_.arm_frame(ps.numpy(), 4, warm=True, layers_out=pl.numpy(), wait_s=5.0)
                if k == 3:
                    with pytest.raises(fw.FewhaError) as ei:
                        S_.solve(4)
                    assert ei.value.name == "STATE"
                ps.numpy()[:] = S_in[k]
                S_.fire_frame()
            dev_s.copy_(torch.from_numpy(S_in[k]).cuda())
            torch.cuda.synchronize()
            B.frame(dev_s, 4, warm=True, layers_out=dev_l)
            B.sync()
            want = dev_l.cpu().numpy()
            for _, pl in bufs:
                assert np.array_equal(pl.numpy(), want), k
            assert rel(want, ref[k][0]) < 1e-4, k


def test_armed_frame_deadline_reported_and_recoverable(fw, elt_frames):
    """An armed frame that is not fired within its deadline does no work and
    reports TIMEOUT (the kernel's wait is bounded); the state is untouched
    and the next frames run normally."""
    import time

    import torch
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as A:
        pin_s = torch.empty(A.S, dtype=torch.float32).pin_memory()
        pin_l = torch.empty(A.N, dtype=torch.float32).pin_memory()
        for k in range(3):
            A.arm_frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy(), wait_s=5.0)
            pin_s.numpy()[:] = S_in[k]
            A.fire_frame()
        state = A.get_state()
        A.arm_frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy(), wait_s=0.002)
        time.sleep(0.1)
        pin_s.numpy()[:] = S_in[3]
        with pytest.raises(fw.FewhaError) as ei:
            A.fire_frame()
        assert ei.value.name == "TIMEOUT"
        for got, want in zip(A.get_state(), state):
            assert np.array_equal(got, want)
        A.set_state(*state, frame_count=3)
        for k in range(3, 5):
            A.arm_frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy(), wait_s=5.0)
            pin_s.numpy()[:] = S_in[k]
            A.fire_frame()
            assert rel(pin_l.numpy(), ref[k][0]) < 1e-4, k


def test_armed_frame_released_when_handle_closes(fw, elt_frames):
    """Closing a handle with a frame still armed fires it (the kernel runs the
    frame instead of holding the GPU until its deadline), so the close returns
    promptly and the next handle works."""
    import time

    import torch
    cfg, S_in, ref = elt_frames
    pin_s = torch.empty(int(sum(2 * w["n_sub"] ** 2 for w in cfg["wfs"])), dtype=torch.float32).pin_memory()
    A = _fused(fw, cfg, k_rr=10)
    pin_l = torch.empty(A.N, dtype=torch.float32).pin_memory()
    assert pin_s.numel() == A.S
    pin_s.numpy()[:] = S_in[0]
    A.arm_frame(pin_s.numpy(), 4, warm=True, layers_out=pin_l.numpy(), wait_s=30.0)
    t0 = time.perf_counter()
    A.close()
    assert time.perf_counter() - t0 < 5.0
    with _fused(fw, cfg, k_rr=10) as B:
        lay = np.empty(B.N, np.float32)
        B.frame(np.ascontiguousarray(S_in[0]), 4, warm=True, layers_out=lay)
        assert rel(lay, ref[0][0]) < 1e-4


def test_fused_graph_frames_on_rotating_buffers(fw, elt_frames):
    """A new slopes and layers buffer every frame, enqueued back to back (the
    cached graph is updated in place, not re-instantiated): the layers are
    bit-identical to frames through fixed buffers, one launch per frame."""
    import torch
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as A, _fused(fw, cfg, k_rr=10) as B:
        fixed_s = torch.empty(A.S, dtype=torch.float32, device="cuda")
        fixed_l = torch.empty(A.N, dtype=torch.float32, device="cuda")
        pool = torch.from_numpy(S_in[:12]).cuda()              # one slopes buffer per frame
        outs = torch.empty(12, B.N, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        l0 = B.launch_count()
        with torch.cuda.stream(B.stream):
            for k in range(12):
                B.frame(pool[k], 4, warm=True, layers_out=outs[k])
        B.sync()
        assert B.launch_count() - l0 == 12
        for k in range(12):
            with torch.cuda.stream(A.stream):
                fixed_s.copy_(pool[k])
            A.frame(fixed_s, 4, warm=True, layers_out=fixed_l)
            A.sync()
            got = outs[k].cpu().numpy()
            assert np.array_equal(got, fixed_l.cpu().numpy()), k
            assert rel(got, ref[k][0]) < 1e-4, k


def test_fused_request_without_plan_refused(fw):
    """A 64 x 64 sensor on 8 x 8 layer grids puts about 8 sensor nodes in every
    layer cell pair, beyond the fused P^T gather's width: the handle runs the
    plain path, and asking for the fused one fails with the reason instead of
    silently keeping the plain path."""
    cfg = configs.tiny(n_sub=64, n=8, levels=(1, 1), G=2, lgs=False, obstruction=0.0, D=4.0)
    with fw.Solver(cfg, precision=fw.FP32) as S:
        assert "path plain" in S.describe()
        with pytest.raises(fw.FewhaError) as ei:
            S.set_path(fw.PATH_FUSED)
        assert ei.value.name == "GEOMETRY" and "sensor grid much finer" in str(ei.value)
        assert "path plain" in S.describe()


@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_fused_every_cluster_shape_matches_oracle(fw, elt_frames, C):
    """Each thread-block-cluster shape of the fused plan (row stripes of n/C
    rows per CTA) gives the same frames as the oracle; shapes that do not fit
    the device are refused with FEWHA_ERR_ARG, never launched."""
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as S:
        try:
            S.set_cluster_size(C)
        except fw.FewhaError as e:
            assert e.code == 1   # FEWHA_ERR_ARG
            pytest.skip("cluster size %d has no plan on this device" % C)
        assert (" x %d CTAs" % C) in S.describe()
        for k in range(11):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            S.sync()
            assert rel(S.layers(), ref[k][0]) < 1e-4, k


def test_fused_autotune_keeps_state_and_parity(fw, elt_frames):
    """The autotuner times candidate plans on the current frame but restores
    the solver state: the frames that follow still match the oracle."""
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as S:
        for k in range(3):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
        rep = S.autotune(n_iter=4, reps=3)
        assert "chosen C=" in rep
        for k in range(3, 12):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            S.sync()
            assert rel(S.layers(), ref[k][0]) < 1e-4, (k, rep)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("name", ["c2_elt", "c1_plain", "ragged"])
def test_both_layer_transforms_match_oracle(fw, name, form):
    """The fused layer phase in each form -- row stripes with a cluster barrier
    per DWT level, and the level-stacked transform with one exchange each way
    -- against the oracle over frames across a residual replacement."""
    cfg = ragged_cfg() if name == "ragged" else configs.ALL[name]()
    nf = 4
    S_in, _ = synth.frames(cfg, nf)
    R = fo.Reconstructor(cfg)
    sides = [l["n"] for l in cfg["layers"]]
    with _fused(fw, cfg, k_rr=3) as S:
        S.set_layer_transform(form)
        assert ("level-stacked" if form else "row stripes") in S.describe()
        for k in range(nf):
            R.frame(S_in[k], 4, warm=True, k_rr=3)
            S.set_frame(S_in[k].astype(np.float32))
            S.solve(4, warm=True)
            S.sync()
            assert rel(S.layers(), R.layers()) < 1e-4, (name, form, k)
            assert rel(S.vector(fw.VEC_C), R.state.c) < 1e-4, (name, form, k)
            elementwise_check(S.layers(), R.layers(), sides, 1e-3, what=(name, form, k))


@pytest.mark.parametrize("C", [4, 8, 16])
def test_level_stacked_transform_every_cluster_shape(fw, elt_frames, C):
    """The level-stacked layer phase on clusters of 4, 8 and 16 (column
    stripes of 32, 16 and 8 columns, different row ownership tables)."""
    cfg, S_in, ref = elt_frames
    with _fused(fw, cfg, k_rr=10) as S:
        S.set_layer_transform(1)
        try:
            S.set_cluster_size(C)
        except fw.FewhaError as e:
            pytest.skip("no plan with clusters of %d: %s" % (C, e))
        assert "level-stacked" in S.describe() and (" x %d CTAs" % C) in S.describe()
        for k in range(3):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            S.sync()
            assert rel(S.layers(), ref[k][0]) < 1e-4, (C, k)
